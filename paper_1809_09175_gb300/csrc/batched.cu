// batched.cu -- MTTKRP of all modes of many tensors in one persistent launch.
//
// Every (tensor, mode) pair is a task; a task's nonzeros (its mode-sorted
// packed records) are cut into chunks of its schedule's npw nonzeros, and all
// chunks of all tasks form one global item space.  A persistent grid of warps
// claims items with an atomic counter (uneven tensors balance themselves),
// stages each item's records with a bulk copy while the previous item is
// computed, and runs the same per-chunk routine as the single-tensor kernel
// (Sec. 6 permuted traversal over sorted nonzeros, Fig. MTTKRP-C).  One
// zero-fill kernel clears every output and the counter first; the two
// launches are captured once in a CUDA graph and replayed.
#include <vector>

#include "internal.h"
#include "mttkrp_kernel.cuh"

namespace spt {
namespace {

struct BatchTask {
    MttkrpParams p;      // M_SORTED parameters of this (tensor, mode)
    int64_t first_item;  // first chunk of this task in the global item space
    int d1;              // order - 1
    int C;               // chunks per lane
};

struct ZeroSeg {
    float *ptr;
    int64_t n;
};

__global__ void batch_zero_kernel(const ZeroSeg *segs, int nseg, unsigned long long *counter) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
    for (int s = blockIdx.y; s < nseg; s += gridDim.y) {
        float4 *p4 = reinterpret_cast<float4 *>(segs[s].ptr);
        const int64_t n4 = segs[s].n / 4;  // outputs are I x ld with ld % 8 == 0
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
             i += (int64_t)gridDim.x * blockDim.x)
            p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ int find_task(const BatchTask *tasks, int ntasks, int64_t item) {
    int lo = 0, hi = ntasks - 1;  // last task with first_item <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].first_item <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename FT, int C, int D1>
__device__ __forceinline__ void run_chunk(const MttkrpParams &p, const int32_t *buf, int n) {
    int b0, b1;
    chunk_bounds<D1, M_SORTED>(p, buf, n, b0, b1);
    mttkrp_chunk<FT, C, D1, M_SORTED>(p, buf, n, b0, b1, nullptr, nullptr);
}

template <typename FT>
__device__ __forceinline__ void run_item(const MttkrpParams &p, int d1, int C, const int32_t *buf, int n) {
    switch (d1 * 2 + C - 1) {
    case 2: run_chunk<FT, 1, 1>(p, buf, n); break;
    case 3: run_chunk<FT, 2, 1>(p, buf, n); break;
    case 4: run_chunk<FT, 1, 2>(p, buf, n); break;
    case 5: run_chunk<FT, 2, 2>(p, buf, n); break;
    case 6: run_chunk<FT, 1, 3>(p, buf, n); break;
    case 7: run_chunk<FT, 2, 3>(p, buf, n); break;
    case 8: run_chunk<FT, 1, 4>(p, buf, n); break;
    case 9: run_chunk<FT, 2, 4>(p, buf, n); break;
    default: break;
    }
}

template <typename FT>
__global__ void __launch_bounds__(256, 2) mttkrp_batch_kernel(const BatchTask *__restrict__ tasks,
                                                             int ntasks, int64_t total,
                                                             unsigned long long *counter,
                                                             int stage_words, int *err) {
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw) + 2 * warp;
    int32_t *wbuf = reinterpret_cast<int32_t *>(smem_raw + 16 * wpc) + (size_t)warp * 2 * stage_words;

    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncwarp();

    auto claim = [&]() -> int64_t {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        return (int64_t)__shfl_sync(FULL, it, 0);
    };
    auto item_len = [&](const BatchTask &tk, int64_t item) {
        const int64_t c0 = (item - tk.first_item) * tk.p.npw;
        const int64_t rem = tk.p.nnz - c0;
        return (int)(rem < tk.p.npw ? rem : tk.p.npw);
    };
    auto issue = [&](int64_t item, int tix, int s) {  // lane 0
        const BatchTask &tk = tasks[tix];
        const int rw = record_words(tk.d1 + 1);
        const int n = item_len(tk, item);
        const int64_t c0 = (item - tk.first_item) * tk.p.npw;
        const uint32_t bytes = (uint32_t)((n * rw) & ~3) * 4u;
        mbar_arrive_expect_tx(&bars[s], bytes);
        if (bytes) bulk_g2s(wbuf + s * stage_words, tk.p.rec + c0 * rw, bytes, &bars[s]);
    };

    int64_t nxt = claim();
    int tix_n = nxt < total ? find_task(tasks, ntasks, nxt) : 0;
    if (nxt < total && lane == 0) issue(nxt, tix_n, 0);
    int k = 0;
    while (nxt < total) {
        const int64_t cur = nxt;
        const int tix = tix_n;
        nxt = claim();
        if (nxt < total) {
            tix_n = find_task(tasks, ntasks, nxt);
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(nxt, tix_n, (k + 1) & 1);
            }
        }
        const int s = k & 1;
        const uint32_t parity = (uint32_t)(k >> 1) & 1u;
        const bool ok = mbar_wait(&bars[s], parity);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicExch(err, SPT_DEV_TIMEOUT);
            if (nxt < total) mbar_wait(&bars[s ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            mbar_wait(&bars[s], parity);
            return;
        }
        const MttkrpParams p = tasks[tix].p;
        const int d1 = tasks[tix].d1, C = tasks[tix].C;
        const int rw = record_words(d1 + 1);
        int32_t *buf = wbuf + s * stage_words;
        const int n = item_len(tasks[tix], cur);
        {  // words past the 16-byte body of a ragged chunk
            const int64_t c0 = (cur - tasks[tix].first_item) * p.npw;
            const int W = n * rw, wb = W & ~3;
            if (lane < W - wb) buf[wb + lane] = __ldg(p.rec + c0 * rw + wb + lane);
        }
        __syncwarp();
        run_item<FT>(p, d1, C, buf, n);
        __syncwarp();  // the stage is free before it is refilled
        ++k;
    }
}

int ilog2i(int x) {
    int r = 0;
    while ((1 << r) < x) ++r;
    return r;
}

}  // namespace
}  // namespace spt

using namespace spt;

struct spt_batch_s {
    spt_dtype fdt = SPT_F32;
    std::vector<BatchTask> htasks;
    std::vector<ZeroSeg> hsegs;
    BatchTask *dtasks = nullptr;
    ZeroSeg *dsegs = nullptr;
    unsigned long long *counter = nullptr;
    int *err = nullptr;
    int64_t total = 0;
    int stage_words = 0;
    int wpc = 8;
    size_t smem = 0;
    int blocks = 0;
    cudaGraphExec_t exec = nullptr;
};

namespace {
spt_status enqueue_batch(spt_batch b, cudaStream_t st) {
    if (b->total == 0) return SPT_OK;
    dim3 zg(64, (unsigned)std::min<size_t>(b->hsegs.size(), 1024));
    batch_zero_kernel<<<zg, 256, 0, st>>>(b->dsegs, (int)b->hsegs.size(), b->counter);
    SPT_LAUNCH_CHECK("batch_zero_kernel");
    const int nt = (int)b->htasks.size();
    if (b->fdt == SPT_F32)
        mttkrp_batch_kernel<float><<<b->blocks, b->wpc * 32, b->smem, st>>>(
            b->dtasks, nt, b->total, b->counter, b->stage_words, b->err);
    else if (b->fdt == SPT_BF16)
        mttkrp_batch_kernel<__nv_bfloat16><<<b->blocks, b->wpc * 32, b->smem, st>>>(
            b->dtasks, nt, b->total, b->counter, b->stage_words, b->err);
    else
        mttkrp_batch_kernel<__half><<<b->blocks, b->wpc * 32, b->smem, st>>>(
            b->dtasks, nt, b->total, b->counter, b->stage_words, b->err);
    SPT_LAUNCH_CHECK("mttkrp_batch_kernel");
    return SPT_OK;
}

template <typename FT> const void *batch_fn() { return (const void *)mttkrp_batch_kernel<FT>; }
}  // namespace

extern "C" {

spt_status mttkrp_batch_create(int count, const spt_batch_item *items, spt_dtype fdt, spt_batch *out) {
    if (!out || (count > 0 && !items)) return fail(SPT_EINVAL, "mttkrp_batch_create: NULL argument");
    *out = nullptr;
    if (count < 0) return fail(SPT_EINVAL, "mttkrp_batch_create: negative count");
    if (fdt == SPT_F64) return fail(SPT_EUNSUPPORTED, "mttkrp_batch_create: fp64 factors are supported by mttkrp only");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16) return fail(SPT_EINVAL, "mttkrp_batch_create: bad dtype");
    spt_batch b = new (std::nothrow) spt_batch_s();
    if (!b) return fail(SPT_ENOMEM, "mttkrp_batch_create: host allocation");
    b->fdt = fdt;
    int64_t first = 0;
    for (int q = 0; q < count; ++q) {
        const spt_batch_item &it = items[q];
        spt_tensor t = it.tensor;
        if (!t || !it.factors || !it.outs) { delete b; return fail(SPT_EINVAL, "mttkrp_batch_create: NULL in item"); }
        if (t->d < 2 || t->d > SPT_MAX_KERNEL_ORDER) { delete b; return fail(SPT_EUNSUPPORTED, "mttkrp_batch_create: order must be in [2, 5]"); }
        if (it.rank < 1 || it.ld < it.rank || it.ld % 8 || it.ld > (1 << 28)) {
            delete b;
            return fail(SPT_EINVAL, "mttkrp_batch_create: bad rank/ld");
        }
        for (int n = 0; n < t->d; ++n) {
            if (it.mode >= 0 && n != it.mode) continue;
            if (!t->sorted_buf[n]) {
                delete b;
                return fail(SPT_ESTATE, "mttkrp_batch_create: every mode needs build_mode_permutation "
                                        "with the mode-sorted copy");
            }
            float *o = it.mode >= 0 ? it.outs[0] : it.outs[n];
            if (!o || ((uintptr_t)o & 15)) { delete b; return fail(SPT_EINVAL, "mttkrp_batch_create: bad output pointer"); }
            spt_schedule sc = default_schedule(t, n, fdt, it.rank);
            if (it.scheds) sc = it.mode >= 0 ? it.scheds[0] : it.scheds[n];
            sc.scatter = SPT_SCATTER_SORTED;
            spt_status cs = check_schedule(t, n, fdt, it.rank, sc);
            if (cs) { delete b; return cs; }
            BatchTask tk{};
            MttkrpParams &p = tk.p;
            const int L = sc.lanes_per_nnz, C = sc.chunks, G = 32 / L;
            int S = std::max(1, sc.nnz_per_group);  // same bank rule as the single kernel
            if (G >= 4) S = (S & 1) ? S : S - 1;
            else if (G == 2) S = std::max(2, (S & ~3) | 2);
            else S = std::max(4, (S + 3) & ~3);
            p.rows = t->idx[n];
            p.vals = t->vals;
            p.perm = t->perm[n];
            p.rec = reinterpret_cast<const int32_t *>(t->sorted_buf[n]);
            int qq = 0;
            for (int m = 0; m < t->d; ++m) {
                if (m == n) continue;
                if (!it.factors[m] || ((uintptr_t)it.factors[m] & 15)) {
                    delete b;
                    return fail(SPT_EINVAL, "mttkrp_batch_create: bad factor pointer");
                }
                p.oidx[qq] = t->idx[m];
                p.fac[qq] = it.factors[m];
                ++qq;
            }
            p.fld = it.ld;
            p.lambda = nullptr;
            p.out = o;
            p.old = it.ld;
            p.nnz = t->nnz;
            p.R = it.rank;
            p.rb_cols = L * C * 4;
            p.n_rb = (it.rank + p.rb_cols - 1) / p.rb_cols;
            p.log2L = ilog2i(L);
            p.S = S;
            p.npw = G * S;
            p.nchunks = (t->nnz + p.npw - 1) / p.npw;
            p.err = nullptr;
            tk.first_item = first;
            tk.d1 = t->d - 1;
            tk.C = C;
            first += p.nchunks;
            b->stage_words = std::max(b->stage_words, (p.npw * record_words(t->d) + 3) & ~3);
            b->htasks.push_back(tk);
            b->hsegs.push_back(ZeroSeg{o, t->dims[n] * (int64_t)it.ld});
        }
    }
    b->total = first;
    b->smem = 16 * (size_t)b->wpc + (size_t)b->wpc * 2 * b->stage_words * 4;
    if (b->smem > 227 * 1024) { delete b; return fail(SPT_EINVAL, "mttkrp_batch_create: staging exceeds shared memory"); }
    const void *fn = fdt == SPT_F32 ? batch_fn<float>() : (fdt == SPT_BF16 ? batch_fn<__nv_bfloat16>() : batch_fn<__half>());
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    int bps = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, b->wpc * 32, b->smem);
    if (e != cudaSuccess || bps < 1) { delete b; return e != cudaSuccess ? cuda_fail(e, "mttkrp_batch_create") : fail(SPT_EINVAL, "batch kernel does not fit"); }
    b->blocks = bps * sm_count();
    // device copies of the task table and zero list, counter, status word
    e = cudaMalloc(&b->dtasks, sizeof(BatchTask) * std::max<size_t>(1, b->htasks.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->dsegs, sizeof(ZeroSeg) * std::max<size_t>(1, b->hsegs.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
    if (e == cudaSuccess && !b->htasks.empty())
        e = cudaMemcpy(b->dtasks, b->htasks.data(), sizeof(BatchTask) * b->htasks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b->hsegs.empty())
        e = cudaMemcpy(b->dsegs, b->hsegs.data(), sizeof(ZeroSeg) * b->hsegs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(b->dtasks); cudaFree(b->dsegs); cudaFree(b->counter); cudaFree(b->err);
        delete b;
        return cuda_fail(e, "mttkrp_batch_create: device tables");
    }
    for (auto &tk : b->htasks) tk.p.err = b->err;
    cudaMemcpy(b->dtasks, b->htasks.data(), sizeof(BatchTask) * b->htasks.size(), cudaMemcpyHostToDevice);
    *out = b;
    return SPT_OK;
}

spt_status mttkrp_batch_run(spt_batch b, void *stream) {
    if (!b) return fail(SPT_EINVAL, "mttkrp_batch_run: NULL batch");
    cudaStream_t st = (cudaStream_t)stream;
    if (st == 0) return enqueue_batch(b, st);
    if (!b->exec) {
        cudaGraph_t g = nullptr;
        SPT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        spt_status s = enqueue_batch(b, st);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (s) { if (g) cudaGraphDestroy(g); return s; }
        if (e != cudaSuccess) return cuda_fail(e, "mttkrp_batch_run: capture");
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "mttkrp_batch_run: instantiate");
    }
    SPT_CUDA(cudaGraphLaunch(b->exec, st));
    return SPT_OK;
}

spt_status mttkrp_batch_info(spt_batch b, int64_t *tasks, int64_t *items, int *blocks) {
    if (!b) return fail(SPT_EINVAL, "mttkrp_batch_info: NULL batch");
    if (tasks) *tasks = (int64_t)b->htasks.size();
    if (items) *items = b->total;
    if (blocks) *blocks = b->blocks;
    return SPT_OK;
}

spt_status mttkrp_batch_check(spt_batch b, void *stream) {
    if (!b) return fail(SPT_EINVAL, "mttkrp_batch_check: NULL batch");
    int h = 0;
    SPT_CUDA(cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    SPT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (h == SPT_DEV_TIMEOUT) return fail(SPT_ETIMEOUT, "a bounded device wait ran out");
    return SPT_OK;
}

spt_status mttkrp_batch_destroy(spt_batch b) {
    if (!b) return fail(SPT_EINVAL, "mttkrp_batch_destroy: NULL batch");
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->dtasks);
    cudaFree(b->dsegs);
    cudaFree(b->counter);
    cudaFree(b->err);
    delete b;
    return SPT_OK;
}

}  // extern "C"

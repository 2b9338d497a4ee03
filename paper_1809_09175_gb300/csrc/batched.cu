// batched.cu -- MTTKRP of all modes of many tensors in one persistent launch.
//
// Every (tensor, mode) pair is a task; a task's nonzeros (its mode-sorted
// packed records) are cut into chunks of its schedule's npw nonzeros, and a
// task's chunks into blocks of BATCH_BLOCK_CHUNKS.  Tasks are grouped by
// kernel class, the chunks per lane C (1 for every rank up to 128 with the
// library's schedules): every class runs one persistent kernel whose warps
// claim blocks with an atomic counter (uneven tensors balance themselves),
// switch on the task's order, and walk each block as a contiguous range with
// the single-tensor kernel's range routine: staged bulk copies, the segmented
// combine and the run carried across the block's chunks (Sec. 6 permuted
// traversal over sorted nonzeros, Fig. MTTKRP-C).  One zero-fill kernel
// clears every output and the counters first; the launches are captured
// once in a CUDA graph and replayed.
#include <vector>

#include "internal.h"
#include "mttkrp_kernel.cuh"

namespace spt {
namespace {

constexpr int BATCH_BLOCK_CHUNKS = 8;  // chunks a warp claims at a time

struct BatchTask {
    MttkrpParams p;       // M_SORTED parameters of this (tensor, mode)
    int64_t first_block;  // first block of this task in its class's block space
    int d1;               // order - 1 of the tensor
};

struct ZeroSeg {
    float *ptr;
    int64_t n;
};

__global__ void batch_zero_kernel(const ZeroSeg *segs, int nseg, unsigned long long *counters, int ncnt) {
    if (blockIdx.x == 0 && blockIdx.y == 0)
        for (int c = threadIdx.x; c < ncnt; c += blockDim.x) counters[c] = 0ull;
    for (int s = blockIdx.y; s < nseg; s += gridDim.y) {
        float4 *p4 = reinterpret_cast<float4 *>(segs[s].ptr);
        const int64_t n4 = segs[s].n / 4;  // outputs are I x ld with ld % 8 == 0
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
             i += (int64_t)gridDim.x * blockDim.x)
            p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ int find_task(const BatchTask *tasks, int ntasks, int64_t blk) {
    int lo = 0, hi = ntasks - 1;  // last task with first_block <= blk
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].first_block <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent kernel of one class (FT, C, orders up to 4 or order 5); each
// block runs the range routine of its task's order (order 5 has a kernel of
// its own: its extra gathers would make the others spill).  Shared memory
// per warp: two barriers (first 16 * wpc bytes), a carry slot of cb bytes,
// two staging buffers of stage_words words each (the largest task of the
// class).
template <typename FT, int C, bool ORDER5>
__global__ void __launch_bounds__(256, C == 1 ? 3 : 2)
    mttkrp_batch_kernel(const BatchTask *__restrict__ tasks, int ntasks, int64_t total_blocks,
                        unsigned long long *counter, int stage_words, int cb) {
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw) + 2 * warp;
    unsigned char *carry = smem_raw + 16 * wpc + (size_t)warp * cb;
    int32_t *wbuf = reinterpret_cast<int32_t *>(smem_raw + 16 * wpc + (size_t)wpc * cb) +
                    (size_t)warp * 2 * stage_words;
    warp_bars_init(bars);
    uint32_t k = 0;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        const int64_t blk = (int64_t)__shfl_sync(FULL, it, 0);
        if (blk >= total_blocks) break;
        const int t = find_task(tasks, ntasks, blk);
        const MttkrpParams &p = tasks[t].p;  // read through the cache, not copied to registers
        const int64_t c0 = (blk - tasks[t].first_block) * BATCH_BLOCK_CHUNKS;
        const int64_t c1 = c0 + BATCH_BLOCK_CHUNKS < p.nchunks ? c0 + BATCH_BLOCK_CHUNKS : p.nchunks;
        bool ok;
        if (ORDER5) {
            ok = mttkrp_range<FT, C, 4, M_SORTED>(p, bars, carry, wbuf, nullptr, (int)c0, (int)c1, k);
        } else {
            switch (tasks[t].d1) {  // warp-uniform
                case 1: ok = mttkrp_range<FT, C, 1, M_SORTED>(p, bars, carry, wbuf, nullptr, (int)c0, (int)c1, k); break;
                case 2: ok = mttkrp_range<FT, C, 2, M_SORTED>(p, bars, carry, wbuf, nullptr, (int)c0, (int)c1, k); break;
                default: ok = mttkrp_range<FT, C, 3, M_SORTED>(p, bars, carry, wbuf, nullptr, (int)c0, (int)c1, k); break;
            }
        }
        if (!ok) return;
    }
}

// One class of tasks: kernel (C, order 5 or not), its task table and launch shape.
struct BatchClass {
    int C = 1;
    bool order5 = false;
    std::vector<BatchTask> htasks;
    BatchTask *dtasks = nullptr;
    int64_t total_blocks = 0;
    int stage_words = 0;
    int cb = 0;
    size_t smem = 0;
    int blocks = 0;
};

template <typename FT> const void *class_fn(int C, bool order5) {
    static const void *tab[2][2] = {
        {(const void *)mttkrp_batch_kernel<FT, 1, false>, (const void *)mttkrp_batch_kernel<FT, 1, true>},
        {(const void *)mttkrp_batch_kernel<FT, 2, false>, (const void *)mttkrp_batch_kernel<FT, 2, true>}};
    return (C >= 1 && C <= 2) ? tab[C - 1][order5 ? 1 : 0] : nullptr;
}

const void *batch_fn(spt_dtype fdt, int C, bool order5) {
    return fdt == SPT_F32    ? class_fn<float>(C, order5)
           : fdt == SPT_BF16 ? class_fn<__nv_bfloat16>(C, order5)
                             : class_fn<__half>(C, order5);
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
    std::vector<BatchClass> classes;
    std::vector<ZeroSeg> hsegs;
    ZeroSeg *dsegs = nullptr;
    unsigned long long *counters = nullptr;  // one per class
    int *err = nullptr;
    int64_t ntasks = 0;
    int64_t total_chunks = 0;
    int wpc = 8;
    cudaGraphExec_t exec = nullptr;
};

namespace {
spt_status enqueue_batch(spt_batch b, cudaStream_t st) {
    if (b->hsegs.empty()) return SPT_OK;
    dim3 zg(64, (unsigned)std::max<size_t>(1, std::min<size_t>(b->hsegs.size(), 1024)));
    batch_zero_kernel<<<zg, 256, 0, st>>>(b->dsegs, (int)b->hsegs.size(), b->counters, (int)b->classes.size());
    SPT_LAUNCH_CHECK("batch_zero_kernel");
    for (size_t c = 0; c < b->classes.size(); ++c) {
        BatchClass &k = b->classes[c];
        const BatchTask *dt = k.dtasks;
        int nt = (int)k.htasks.size();
        int64_t tb = k.total_blocks;
        unsigned long long *cnt = b->counters + c;
        int sw = k.stage_words, cb = k.cb;
        void *args[] = {(void *)&dt, (void *)&nt, (void *)&tb, (void *)&cnt, (void *)&sw, (void *)&cb};
        SPT_CUDA(cudaLaunchKernel(batch_fn(b->fdt, k.C, k.order5), dim3(k.blocks), dim3(b->wpc * 32), args, k.smem, st));
    }
    return SPT_OK;
}

void free_batch(spt_batch b) {
    for (auto &k : b->classes) cudaFree(k.dtasks);
    cudaFree(b->dsegs);
    cudaFree(b->counters);
    cudaFree(b->err);
    delete b;
}
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
            // one class kernel serves every task, and its staging is sized for
            // the largest chunk: cap each task's chunk at the default rule's
            // 6 KB of shared memory per warp, so one task with long chunks
            // does not cut the occupancy of the whole batch
            const int npw_cap = std::max(G, (6144 - 16 - carry_bytes(C, L, 4)) / (8 * record_words(t->d)));
            int S = std::max(1, std::min(sc.nnz_per_group, std::max(1, npw_cap / G)));  // same bank rule as the single kernel
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
            p.loss = -1;
            b->hsegs.push_back(ZeroSeg{o, t->dims[n] * (int64_t)it.ld});
            ++b->ntasks;
            if (t->nnz == 0) continue;  // zero-filled, nothing to add
            tk.d1 = t->d - 1;
            const bool o5 = t->d == 5;
            BatchClass *cls = nullptr;
            for (auto &k : b->classes)
                if (k.C == C && k.order5 == o5) cls = &k;
            if (!cls) {
                b->classes.emplace_back();
                cls = &b->classes.back();
                cls->C = C;
                cls->order5 = o5;
            }
            tk.first_block = cls->total_blocks;
            cls->total_blocks += (p.nchunks + BATCH_BLOCK_CHUNKS - 1) / BATCH_BLOCK_CHUNKS;
            cls->stage_words = std::max(cls->stage_words, p.npw * record_words(t->d));
            cls->cb = std::max(cls->cb, carry_bytes(C, L, 4));
            b->total_chunks += p.nchunks;
            cls->htasks.push_back(tk);
        }
    }
    cudaError_t e = cudaMalloc(&b->counters, sizeof(unsigned long long) * std::max<size_t>(1, b->classes.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->dsegs, sizeof(ZeroSeg) * std::max<size_t>(1, b->hsegs.size()));
    if (e == cudaSuccess && !b->hsegs.empty())
        e = cudaMemcpy(b->dsegs, b->hsegs.data(), sizeof(ZeroSeg) * b->hsegs.size(), cudaMemcpyHostToDevice);
    for (auto &k : b->classes) {
        if (e != cudaSuccess) break;
        k.stage_words = (k.stage_words + 3) & ~3;  // 16-byte aligned staging buffers
        k.smem = 16 * (size_t)b->wpc + (size_t)b->wpc * k.cb + (size_t)b->wpc * 2 * k.stage_words * 4;
        if (k.smem > 227 * 1024) { free_batch(b); return fail(SPT_EINVAL, "mttkrp_batch_create: staging exceeds shared memory"); }
        const void *fn = batch_fn(fdt, k.C, k.order5);
        if (!fn) { free_batch(b); return fail(SPT_EUNSUPPORTED, "mttkrp_batch_create: no kernel for this class"); }
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
        int bps = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, b->wpc * 32, k.smem);
        if (e == cudaSuccess && bps < 1) { free_batch(b); return fail(SPT_EINVAL, "batch kernel does not fit"); }
        k.blocks = bps * sm_count();
        for (auto &tk : k.htasks) {
            tk.p.err = b->err;
            tk.p.wait_tries = wait_tries();
        }
        if (e == cudaSuccess) e = cudaMalloc(&k.dtasks, sizeof(BatchTask) * std::max<size_t>(1, k.htasks.size()));
        if (e == cudaSuccess)
            e = cudaMemcpy(k.dtasks, k.htasks.data(), sizeof(BatchTask) * k.htasks.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "mttkrp_batch_create: device tables");
    }
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
    if (tasks) *tasks = b->ntasks;
    if (items) *items = b->total_chunks;
    if (blocks) {
        int m = 0;
        for (auto &k : b->classes) m = std::max(m, k.blocks);
        *blocks = m;
    }
    return SPT_OK;
}

spt_status mttkrp_batch_check(spt_batch b, void *stream) {
    if (!b) return fail(SPT_EINVAL, "mttkrp_batch_check: NULL batch");
    int h = 0;
    SPT_CUDA(cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    SPT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (h) {  // reported once: clear the word for the runs that follow
        SPT_CUDA(cudaMemsetAsync(b->err, 0, sizeof(int), (cudaStream_t)stream));
        SPT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    }
    if (h == SPT_DEV_TIMEOUT) return fail(SPT_ETIMEOUT, "a bounded device wait ran out");
    if (h) return fail(SPT_ECUDA, "device status word " + std::to_string(h));
    return SPT_OK;
}

spt_status mttkrp_batch_destroy(spt_batch b) {
    if (!b) return fail(SPT_EINVAL, "mttkrp_batch_destroy: NULL batch");
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    free_batch(b);
    return SPT_OK;
}

}  // extern "C"

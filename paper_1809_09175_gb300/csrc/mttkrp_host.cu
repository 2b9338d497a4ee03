// mttkrp_host.cu -- schedule logic and launch of the MTTKRP kernel.
#include <atomic>
#include <cmath>
#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "mttkrp_kernel.cuh"

// Shared-memory bytes of the atomic scatter's per-CTA copy of the hot rows
// (R = 16 fp32: 256 rows; R = 64: 64 rows).
#ifndef SPT_HOT_SMEM
#define SPT_HOT_SMEM (16 * 1024)
#endif
// Atomic scatter: the estimated relative error of the adds above which they
// are split over copies of the output (a third of the 1e-5 fp32 gate), at
// most SPT_ATOMIC_COPIES_MAX copies of at most SPT_ATOMIC_COPY_BYTES in all.
#ifndef SPT_ATOMIC_COPY_EST
#define SPT_ATOMIC_COPY_EST 3e-6
#endif
#ifndef SPT_ATOMIC_COPIES_MAX
#define SPT_ATOMIC_COPIES_MAX 64
#endif
#ifndef SPT_ATOMIC_COPY_BYTES
#define SPT_ATOMIC_COPY_BYTES (512ll << 20)
#endif

// 0: never take the clamped-gather kernels (build variant for comparisons)
#ifndef SPT_CLAMP_GATHERS
#define SPT_CLAMP_GATHERS 1
#endif

namespace spt {

namespace {
std::atomic<uint32_t> g_wait_tries{SPT_WAIT_TRIES};
}
uint32_t wait_tries() { return g_wait_tries.load(std::memory_order_relaxed); }

int elem_bytes(spt_dtype fdt) { return fdt == SPT_F64 ? 8 : (fdt == SPT_F32 ? 4 : 2); }
int acc_bytes(spt_dtype fdt) { return fdt == SPT_F64 ? 8 : 4; }

namespace {
// Deterministic sums: out(row, :) = the sum of the slots holding `row` (slot
// rows are non-decreasing where set, -1 where unused; a row held by a slot
// receives no other write).  One warp per slot i, working when i starts its
// row's run of slots: a run of at most 8 slots is added in slot order, one
// lane per column quad; a longer run (a hot row spread over many warps'
// ranges) is split over the lanes (lane t takes slots i+t, i+t+32, ...) and
// the lanes' sums are combined by a fixed shuffle tree.  The order of every
// addition depends on the slot layout only, never on timing.
template <typename AT>
__global__ void __launch_bounds__(256) det_fixup_kernel(const int *__restrict__ rows, const AT *__restrict__ vals,
                                                        int nslots, int R, int64_t old, AT *out) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int q4 = (R + 3) / 4;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nslots; i += nw) {
        const int row = rows[i];  // warp-uniform from here on
        if (row < 0) continue;
        int prev = i - 1;
        while (prev >= 0 && rows[prev] < 0) --prev;
        if (prev >= 0 && rows[prev] == row) continue;  // not the first slot of this row
        int end = nslots;  // the first slot past i holding another row
        for (int k0 = i + 1; k0 < nslots; k0 += 32) {
            const int k = k0 + lane;
            const int rk = k < nslots ? rows[k] : -1;
            const unsigned b = __ballot_sync(FULL, rk >= 0 && rk != row);
            if (b) {
                end = k0 + __ffs(b) - 1;
                break;
            }
        }
        AT *dst = out + (int64_t)row * old;
        if (end - i <= 8) {
            for (int q = lane; q < q4; q += 32) {
                AT sum[4] = {(AT)0, (AT)0, (AT)0, (AT)0};
                for (int k = i; k < end; ++k) {
                    if (rows[k] != row) continue;  // an unused slot
#pragma unroll
                    for (int v = 0; v < 4; ++v) sum[v] += vals[(int64_t)k * old + 4 * q + v];
                }
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (4 * q + v < R) dst[4 * q + v] = sum[v];
            }
            continue;
        }
        for (int q = 0; q < q4; ++q) {
            AT sum[4] = {(AT)0, (AT)0, (AT)0, (AT)0};
            for (int k = i + lane; k < end; k += 32) {
                if (rows[k] != row) continue;
#pragma unroll
                for (int v = 0; v < 4; ++v) sum[v] += vals[(int64_t)k * old + 4 * q + v];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int v = 0; v < 4; ++v) sum[v] += __shfl_down_sync(FULL, sum[v], o);
            if (lane == 0) {
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (4 * q + v < R) dst[4 * q + v] = sum[v];
            }
        }
    }
}

// Deterministic sums: the kernel writes the two boundary rows of each warp's
// range (row id, partial row) into slots 2w and 2w+1 of a scratch array;
// det_fixup_kernel then stores each such row as the sum of its slots.  Every
// other row has one writer, so the result does not depend on the order in
// which warps finish.
spt_status launch_det(MttkrpKernelFn fn, MttkrpParams p, int blocks, int wpc, size_t smem, int ab,
                      cudaStream_t st) {
    const int nslots = 2 * blocks * wpc;
    const size_t rows_bytes = ((size_t)nslots * sizeof(int) + 255) & ~(size_t)255;
    void *buf = nullptr;
    spt_status c = dmalloc(&buf, rows_bytes + (size_t)nslots * p.old * ab, st);
    if (c) return c;
    p.det_rows = reinterpret_cast<int *>(buf);
    p.det_vals = reinterpret_cast<char *>(buf) + rows_bytes;
    cudaError_t e = cudaMemsetAsync(p.det_rows, 0xff, (size_t)nslots * sizeof(int), st);  // -1: unused
    if (e == cudaSuccess) {
        fn<<<blocks, wpc * 32, smem, st>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int fb = std::max(1, std::min((nslots + 7) / 8, sm_count() * 16));  // a warp per slot
        if (ab == 8)
            det_fixup_kernel<double><<<fb, 256, 0, st>>>(p.det_rows, (const double *)p.det_vals, nslots, p.R, p.old,
                                                         (double *)p.out);
        else
            det_fixup_kernel<float><<<fb, 256, 0, st>>>(p.det_rows, (const float *)p.det_vals, nslots, p.R, p.old,
                                                        (float *)p.out);
        e = cudaGetLastError();
    }
    dfree(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp deterministic launch");
    return SPT_OK;
}

// out[i] = the sum of the nrep copies scratch[r * n + i] (fp64 sum, one rounding)
template <typename AT>
__global__ void sum_copies_kernel(const AT *__restrict__ scratch, int nrep, int64_t n, AT *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int r = 0; r < nrep; ++r) a += (double)scratch[(int64_t)r * n + i];
        out[i] = (AT)a;
    }
}

// Atomic scatter into nrep zeroed copies of the output (stream-ordered
// scratch; CTA b adds into copy b mod nrep), summed into the output after.
// Each copy takes 1/nrep of every row's adds, so each chain of fp32 adds is
// nrep times shorter and its partial sums nrep times smaller.
spt_status launch_copies(MttkrpKernelFn fn, MttkrpParams p, int blocks, int wpc, size_t smem, int64_t In, int ab,
                         cudaStream_t st) {
    const int64_t n = In * p.old;
    void *buf = nullptr;
    spt_status c = dmalloc(&buf, (size_t)ab * (size_t)n * p.nrep, st);
    if (c) return c;
    void *out = p.out;
    p.out = buf;
    p.rep_stride = n;
    cudaError_t e = cudaMemsetAsync(buf, 0, (size_t)ab * (size_t)n * p.nrep, st);
    if (e == cudaSuccess) {
        fn<<<blocks, wpc * 32, smem, st>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8));
        if (ab == 8)
            sum_copies_kernel<double><<<g, 256, 0, st>>>((const double *)buf, p.nrep, n, (double *)out);
        else
            sum_copies_kernel<float><<<g, 256, 0, st>>>((const float *)buf, p.nrep, n, (float *)out);
        e = cudaGetLastError();
    }
    dfree(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp atomic scatter into copies");
    return SPT_OK;
}

int ilog2(int x) {
    int r = 0;
    while ((1 << r) < x) ++r;
    return r;
}

bool pow2_in(int x, int lo, int hi) { return x >= lo && x <= hi && (x & (x - 1)) == 0; }

// Nonzeros per group, adjusted so that the G groups of a warp read their
// staged elements g*S + t from distinct shared-memory banks and npw = G*S is
// a multiple of 4 (16-byte bulk copies): S odd for G >= 4, S = 2 mod 4 for
// G = 2, S a multiple of 4 for G = 1.
int adjust_S(int want, int G) {
    int S = std::max(1, want);
    if (G >= 4) return (S & 1) ? S : S - 1;  // round down to odd
    if (G == 2) return std::max(2, (S & ~3) | 2);
    return std::max(4, (S + 3) & ~3);
}

std::mutex g_attr_mu;
std::unordered_map<const void *, int> g_attr_smem;

spt_status ensure_smem_attr(MttkrpKernelFn fn, int smem) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int &cur = g_attr_smem[(const void *)fn];
    if (cur >= smem) return SPT_OK;
    SPT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cur = smem;
    return SPT_OK;
}
}  // namespace

size_t schedule_warp_smem(spt_tensor t, const spt_schedule &s, spt_dtype fdt) {
    const int G = 32 / s.lanes_per_nnz;
    const int npw = G * adjust_S(s.nnz_per_group, G);
    const int wpe = s.scatter == SPT_SCATTER_PERM     ? 1
                    : s.scatter == SPT_SCATTER_SORTED ? record_words(t->d)
                                                      : t->d + 1;
    return warp_smem_bytes(s.warps_per_cta, s.chunks, s.lanes_per_nnz, acc_bytes(fdt), wpe, npw);
}

int private_cluster_log2(int64_t In, int rank, size_t warp_smem, int ab) {
    const size_t pld = (size_t)((rank + 3) & ~3);
    for (int k = 0; k <= 3; ++k) {
        const size_t rows = (size_t)((In + (1 << k) - 1) >> k);
        if (warp_smem + rows * pld * ab <= 227 * 1024) return k;
    }
    return -1;
}

spt_schedule default_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank) {
    if (t->pref_set[mode] && t->pref_rank[mode] == rank && t->pref_fdt[mode] == fdt &&
        check_schedule(t, mode, fdt, rank, t->pref[mode]) == SPT_OK)
        return t->pref[mode];
    spt_schedule s{};
    s.scatter = t->sorted_buf[mode] ? SPT_SCATTER_SORTED
                                    : (t->perm[mode] ? SPT_SCATTER_PERM : SPT_SCATTER_ATOMIC);
    const int vec = 4;  // columns per lane chunk
    const int need = (rank + vec - 1) / vec;
    int lanes = 1;
    while (lanes < need && lanes < 32) lanes <<= 1;
    s.lanes_per_nnz = lanes;
    s.chunks = need > 32 ? 2 : 1;
    // at most 6 KB of shared memory per warp (barriers, run carry, two
    // staging buffers): four 8-warp CTAs then fit the 196 KB shared-memory
    // carve-out and leave ~60 KB of the SM's L1 for factor-row hits (with
    // 7 KB the 228 KB carve-out leaves 28 KB and the 3-way 1e8 MTTKRP runs
    // 20% slower); at most 256 nonzeros per chunk
    const int narr = s.scatter == SPT_SCATTER_PERM ? 1
                     : (s.scatter == SPT_SCATTER_SORTED ? record_words(t->d) : t->d + 1);
    const int npw = std::min(256, (6144 - 16 - carry_bytes(s.chunks, lanes, acc_bytes(fdt))) / (8 * narr));
    s.nnz_per_group = std::max(4, npw / (32 / lanes));
    s.warps_per_cta = 8;
    s.ctas_per_sm = 0;
    return s;
}

spt_status check_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank, const spt_schedule &s) {
    (void)fdt;
    if (s.scatter < SPT_SCATTER_ATOMIC || s.scatter > SPT_SCATTER_PRIVATE)
        return fail(SPT_EINVAL, "schedule: unknown scatter strategy");
    if (!pow2_in(s.lanes_per_nnz, 1, 32)) return fail(SPT_EINVAL, "schedule: lanes_per_nnz must be 1,2,4,..,32");
    if (s.chunks < 1 || s.chunks > 2) return fail(SPT_EINVAL, "schedule: chunks must be 1 or 2");
    if (s.nnz_per_group < 1 || s.nnz_per_group > 4096) return fail(SPT_EINVAL, "schedule: nnz_per_group in [1, 4096]");
    if (s.warps_per_cta < 1 || s.warps_per_cta > 16) return fail(SPT_EINVAL, "schedule: warps_per_cta in [1, 16]");
    if (s.ctas_per_sm < 0 || s.ctas_per_sm > 32) return fail(SPT_EINVAL, "schedule: ctas_per_sm in [0, 32]");
    if (s.scatter == SPT_SCATTER_PERM && !t->perm[mode])
        return fail(SPT_ESTATE, "schedule: permuted traversal needs build_mode_permutation(mode)");
    if (s.scatter == SPT_SCATTER_SORTED && !t->sorted_buf[mode])
        return fail(SPT_ESTATE, "schedule: sorted traversal needs the mode-sorted copy");
    if (s.scatter == SPT_SCATTER_PRIVATE &&
        private_cluster_log2(t->dims[mode], rank, schedule_warp_smem(t, s, fdt), acc_bytes(fdt)) < 0)
        return fail(SPT_EINVAL, "schedule: the private scatter's copy of this mode's output does not fit "
                                "the shared memory of a cluster of 8 CTAs");
    return SPT_OK;
}

spt_status launch_mttkrp(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                         int rank, int ld, const void *lambda, void *out,
                         const spt_schedule &s, cudaStream_t st, const GcpArgs *gcp, bool det) {
    const int vec = 4;  // columns per lane chunk
    const int L = s.lanes_per_nnz, C = s.chunks;
    const int G = 32 / L;
    const int rb_cols = L * C * vec;
    const int S = adjust_S(s.nnz_per_group, G);
    const int npw = G * S;
    const int wpc = s.warps_per_cta;
    const int ab = acc_bytes(fdt);
    SPT_CUDA(cudaMemsetAsync(out, 0, (size_t)ab * (size_t)t->dims[mode] * ld, st));
    if (t->nnz == 0) return SPT_OK;

    const int D1 = t->d - 1;
    const int kmode = s.scatter == SPT_SCATTER_ATOMIC    ? M_ATOMIC
                      : s.scatter == SPT_SCATTER_SORTED  ? M_SORTED
                      : s.scatter == SPT_SCATTER_PRIVATE ? M_PRIVATE
                                                         : M_PERM;
    MttkrpParams p{};
    p.rows = t->idx[mode];
    p.vals = t->vals;
    p.perm = t->perm[mode];
    p.rec = kmode == M_PERM ? t->srec : reinterpret_cast<const int32_t *>(t->sorted_buf[mode]);
    p.mode = mode;
    int q = 0;
    for (int m = 0; m < t->d; ++m) {
        if (m == mode) continue;
        p.oidx[q] = t->idx[m];
        p.fac[q] = factors[m];
        ++q;
    }
    p.fld = ld;
    p.lambda = lambda;
    p.out = out;
    p.old = ld;
    p.nnz = t->nnz;
    p.R = rank;
    p.rb_cols = rb_cols;
    p.n_rb = (rank + rb_cols - 1) / rb_cols;
    p.log2L = ilog2(L);
    p.S = S;
    p.npw = npw;
    p.nchunks = (t->nnz + npw - 1) / npw;
    p.err = t->dev_err;
    p.wait_tries = wait_tries();
    p.loss = -1;
    if (gcp) {
        if (kmode != M_SORTED || p.n_rb != 1)
            return fail(SPT_EINVAL, "gcp: needs the sorted traversal and one rank block covering the rank");
        p.fac_n = gcp->fac_n;
        p.loss = gcp->loss;
        p.loss_out = gcp->loss_out;
    }
    if (det && (gcp || kmode != M_SORTED || p.n_rb != 1))
        return fail(SPT_EINVAL, "mttkrp: deterministic sums need the sorted traversal and one rank block");

    const int wpe = kmode == M_PERM ? 1 : (kmode == M_SORTED ? record_words(t->d) : D1 + 2);
    size_t smem = warp_smem_bytes(wpc, C, L, ab, wpe, npw);
    if (smem > 227 * 1024)
        return fail(SPT_EINVAL, "schedule: staging buffers exceed 227 KB of shared memory "
                                "(lower warps_per_cta or nnz_per_group)");
    if (kmode == M_ATOMIC && t->nhot[mode] > 0) {
        // the mode's hottest rows go to a shared-memory copy per CTA: at most
        // SPT_HOT_SMEM bytes of accumulators, and never past the 227 KB limit
        const int pld = (rank + 3) & ~3;
        int nhot = (int)std::min<int64_t>(t->nhot[mode], SPT_HOT_SMEM / ((int64_t)pld * ab));
        auto log2T = [](int h) { return std::max(1, ilog2(2 * h)); };
        while (nhot > 0 && smem + hot_smem_bytes(nhot, pld, ab, log2T(nhot)) > 227 * 1024) nhot >>= 1;
        if (nhot > 0) {
            p.hot_rows = t->hot_buf + (size_t)mode * SPT_HOT_MAX;
            p.nhot = nhot;
            p.hot_log2T = log2T(nhot);
            p.pld = pld;
            smem += hot_smem_bytes(nhot, pld, ab, p.hot_log2T);
        }
    }
    // fp32 atomic adds drift along long chains: a row past the hot list takes
    // one add per nonzero (count_k adds), a relative error of about
    // 2^-24 sqrt(count_k) while the rounding errors stay random (more once
    // the partial sums dwarf the terms), i.e. over the output about
    //   2^-24 sqrt(sum_k count_k^3 / sum_all count^2)
    // (rows weighted by their share of ||V||^2, nonnegative terms).  Twice
    // that, above SPT_ATOMIC_COPY_EST, splits the adds over nrep copies of
    // the output (error / nrep or better), as many as SPT_ATOMIC_COPY_BYTES
    // and the grid allow.
    p.nrep = 1;
    p.rep_stride = 0;
    if (kmode == M_ATOMIC && t->cnt_s2[mode] > 0.0) {
        double s3 = t->cnt_s3[mode];
        for (int q = 0; q < p.nhot; ++q) {
            const double c = (double)t->hot_count[mode][q];
            s3 -= c * c * c;
        }
        const double est = 2.0 * std::ldexp(1.0, ab == 4 ? -24 : -53) * std::sqrt(std::max(0.0, s3) / t->cnt_s2[mode]);
        const double copy_bytes = (double)t->dims[mode] * p.old * ab;
        while (p.nrep < SPT_ATOMIC_COPIES_MAX && est / p.nrep > SPT_ATOMIC_COPY_EST &&
               copy_bytes * 2 * p.nrep <= (double)SPT_ATOMIC_COPY_BYTES)
            p.nrep *= 2;
    }
    int K = 1;
    if (kmode == M_PRIVATE) {
        const int log2K = private_cluster_log2(t->dims[mode], rank, smem, ab);
        if (log2K < 0)
            return fail(SPT_EINVAL, "schedule: the private scatter's copy of this mode's output does not fit "
                                    "the shared memory of a cluster of 8 CTAs");
        K = 1 << log2K;
        p.In = (int)t->dims[mode];
        p.pld = (rank + 3) & ~3;
        p.log2K = log2K;
        p.prows = (int)((t->dims[mode] + K - 1) / K);
        smem += (size_t)p.prows * p.pld * ab;
    }
    // A private copy takes every add of its cluster's nonzeros to a row in
    // one chain (count_k / clusters adds, the same fp32 drift as the atomic
    // scatter's): waves of more clusters than fit at once, each over fewer
    // nonzeros, shorten those chains, the estimate over the resident
    // clusters above SPT_ATOMIC_COPY_EST doubling the waves (at most 64).
    int waves = 1;
    double priv_est = 0.0;
    if (kmode == M_PRIVATE && t->cnt_s2[mode] > 0.0)
        priv_est = 2.0 * std::ldexp(1.0, ab == 4 ? -24 : -53) * std::sqrt(t->cnt_s3[mode] / t->cnt_s2[mode]);
    // a lane whose whole chunk lies past column R: with at most 8 lanes per
    // nonzero the sorted traversal takes the clamped-gather kernels, whose
    // gathers then do not diverge (measured: 4-way R=20 1.55x, 5-way R=20
    // 1.12x); with 16 or 32 lanes the predicated gathers were as fast or
    // faster (4-way R=40: 7%, the uniform 3-way R=40..56: 10%)
    const bool idle_chunks = SPT_CLAMP_GATHERS && L <= 8 && (int64_t)p.n_rb * rb_cols - rank >= vec;
    MttkrpKernelFn fn = gcp                 ? gcp_kernel_fn(fdt, C, D1)
                        : det               ? (fdt == SPT_F32    ? mttkrp_kernel_f32_det(C, D1)
                                               : fdt == SPT_BF16 ? mttkrp_kernel_bf16_det(C, D1)
                                               : fdt == SPT_F64  ? mttkrp_kernel_f64_det(C, D1)
                                                                 : mttkrp_kernel_f16_det(C, D1))
                        : (kmode == M_SORTED && idle_chunks)
                            ? (fdt == SPT_F32    ? mttkrp_kernel_f32_clamp(C, D1)
                               : fdt == SPT_BF16 ? mttkrp_kernel_bf16_clamp(C, D1)
                               : fdt == SPT_F64  ? mttkrp_kernel_f64_clamp(C, D1)
                                                 : mttkrp_kernel_f16_clamp(C, D1))
                        : fdt == SPT_F32    ? mttkrp_kernel_f32(C, D1, kmode)
                        : fdt == SPT_BF16   ? mttkrp_kernel_bf16(C, D1, kmode)
                        : fdt == SPT_F64    ? mttkrp_kernel_f64(C, D1, kmode)
                                            : mttkrp_kernel_f16(C, D1, kmode);
    if (!fn) return fail(SPT_EUNSUPPORTED, "mttkrp: no kernel for this order/chunks");
    spt_status e = ensure_smem_attr(fn, (int)smem);
    if (e) return e;
    if (K > 1) {
        // clusters of K CTAs; a persistent grid of as many clusters as fit at once
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(wpc * 32);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(K * sm_count());
        int ncl = 0;
        SPT_CUDA(cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg));
        if (ncl < 1) return fail(SPT_EINVAL, "schedule: a cluster of the private scatter does not fit the GPU");
        const int64_t need_cl = ((p.nchunks + wpc - 1) / wpc + K - 1) / K;
        while (waves < 64 && priv_est / ((double)ncl * waves) > SPT_ATOMIC_COPY_EST && (int64_t)ncl * waves < need_cl)
            waves *= 2;
        const int cl = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ncl * waves, need_cl));
        cfg.gridDim = dim3(cl * K);
        SPT_CUDA(cudaLaunchKernelEx(&cfg, fn, p));
        SPT_LAUNCH_CHECK("mttkrp_kernel cluster launch");
        return SPT_OK;
    }
    int bps = 0;
    SPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, wpc * 32, smem));
    if (bps < 1) return fail(SPT_EINVAL, "schedule: kernel does not fit on an SM");
    const int cps = s.ctas_per_sm > 0 ? std::min(s.ctas_per_sm, bps) : bps;
    const int64_t need = (p.nchunks + wpc - 1) / wpc;
    while (waves < 64 && priv_est / ((double)cps * sm_count() * waves) > SPT_ATOMIC_COPY_EST &&
           (int64_t)cps * sm_count() * waves < need)
        waves *= 2;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)cps * sm_count() * waves, need));
    if (kmode == M_SORTED && !gcp && !det && t->blk_buf[mode]) {
        // the L2-blocked copy: one launch per group of records (one block of
        // the blocked mode's rows), each adding the rows it owns
        const std::vector<int64_t> &off = t->blk_off[mode];
        const int rw = record_words(t->d);
        p.accum = 1;
        for (size_t b = 0; b + 1 < off.size(); ++b) {
            const int64_t nb = off[b + 1] - off[b];
            if (nb == 0) continue;
            p.rec = reinterpret_cast<const int32_t *>(t->blk_buf[mode]) + off[b] * rw;
            p.nnz = nb;
            p.nchunks = (nb + npw - 1) / npw;
            const int64_t nd = (p.nchunks + wpc - 1) / wpc;
            const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)cps * sm_count(), nd));
            fn<<<bl, wpc * 32, smem, st>>>(p);
            SPT_LAUNCH_CHECK("mttkrp_kernel launch (L2-blocked copy)");
        }
        return SPT_OK;
    }
    if (det) return launch_det(fn, p, blocks, wpc, smem, ab, st);
    if (p.nrep > 1) {
        while (p.nrep > 1 && p.nrep > blocks) p.nrep >>= 1;  // a copy per CTA at most
        if (p.nrep > 1) return launch_copies(fn, p, blocks, wpc, smem, t->dims[mode], ab, st);
    }
    fn<<<blocks, wpc * 32, smem, st>>>(p);
    SPT_LAUNCH_CHECK("mttkrp_kernel launch");
    return SPT_OK;
}

}  // namespace spt

extern "C" spt_status spt_set_wait_tries(int64_t tries) {
    if (tries < -1 || tries > (int64_t)UINT32_MAX)
        return spt::fail(SPT_EINVAL, "spt_set_wait_tries: tries must be -1 (default) or in [0, 2^32 - 1]");
    spt::g_wait_tries.store(tries < 0 ? SPT_WAIT_TRIES : (uint32_t)tries, std::memory_order_relaxed);
    return SPT_OK;
}

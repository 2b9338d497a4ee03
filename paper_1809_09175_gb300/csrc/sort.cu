// sort.cu -- mode permutations (Sec. 6), duplicate coalescing (Sec. 3 COO)
// and per-mode slice statistics, built on an on-device stable LSD radix sort.
//
// The paper builds its permutations with library sorts (Thrust, Kokkos); this
// file has its own: per 8-bit digit, (1) a per-tile digit histogram, (2) an
// exclusive scan of the digit-major histogram (digit d of tile t lands after
// every smaller digit and after digit d of every earlier tile), (3) a stable
// scatter in which each warp ranks its items with __match_any_sync and the
// warps of a tile are ordered by a shared-memory prefix.  Tiles, warps,
// rounds and lanes all follow position order, so equal keys keep their order.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "mttkrp_kernel.cuh"

namespace spt {

namespace {
constexpr int SCAN_T = 512, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;
constexpr int RT = 256, RITEMS = 8, RTILE = RT * RITEMS, RWARP_ITEMS = 32 * RITEMS;
constexpr unsigned FULL = 0xffffffffu;

__global__ void scan_block_kernel(const int32_t *in, int32_t *out, int64_t n, int32_t *bsum) {
    __shared__ int32_t wsum[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_I;
    int32_t v[SCAN_I];
    int32_t tot = 0;
#pragma unroll
    for (int q = 0; q < SCAN_I; ++q) {
        const int64_t i = base + q;
        v[q] = (i < n) ? in[i] : 0;
        tot += v[q];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t s = (lane < SCAN_T / 32) ? wsum[lane] : 0;
        int32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(FULL, si, o);
            if (lane >= o) si += y;
        }
        if (lane < SCAN_T / 32) wsum[lane] = si - s;  // exclusive
        if (lane == SCAN_T / 32 - 1) bsum[blockIdx.x] = si;
    }
    __syncthreads();
    int32_t run = wsum[w] + inc - tot;
#pragma unroll
    for (int q = 0; q < SCAN_I; ++q) {
        const int64_t i = base + q;
        if (i < n) out[i] = run;
        run += v[q];
    }
}

__global__ void scan_add_kernel(int32_t *out, int64_t n, const int32_t *boff) {
    const int32_t add = boff[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int q = threadIdx.x; q < SCAN_TILE; q += SCAN_T) {
        const int64_t i = base + q;
        if (i < n) out[i] += add;
    }
}

__global__ void radix_hist_kernel(const uint32_t *keys, int64_t n, int shift, int32_t *hist,
                                  int64_t ntiles) {
    __shared__ int32_t cnt[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RTILE;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < RITEMS; ++r) {
        const int64_t i = base + r * RT + threadIdx.x;
        const bool valid = i < n;
        const uint32_t dg = valid ? ((keys[i] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(FULL, dg);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[dg], __popc(peers));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[(int64_t)t * ntiles + blockIdx.x] = cnt[t];
}

__global__ void radix_scatter_kernel(const uint32_t *kin, const int32_t *vin, int64_t n, int shift,
                                     const int32_t *offs, int64_t ntiles, uint32_t *kout,
                                     int32_t *vout) {
    __shared__ int32_t wcnt[RT / 32][256];
    __shared__ int32_t base[256];
    for (int t = threadIdx.x; t < (RT / 32) * 256; t += blockDim.x) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = (int64_t)blockIdx.x * RTILE + w * RWARP_ITEMS;
    uint32_t key[RITEMS];
    int32_t val[RITEMS], rank[RITEMS];
    uint32_t dgt[RITEMS];
#pragma unroll
    for (int r = 0; r < RITEMS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? (vin ? vin[i] : (int32_t)i) : 0;
        const uint32_t dg = valid ? ((key[r] >> shift) & 255u) : 256u;
        dgt[r] = dg;
        const unsigned peers = __match_any_sync(FULL, dg);
        const int lower = __popc(peers & lt);
        const int running = valid ? wcnt[w][dg] : 0;
        __syncwarp();
        if (valid && lower == 0) wcnt[w][dg] = running + __popc(peers);
        __syncwarp();
        rank[r] = running + lower;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        int32_t s = 0;
#pragma unroll
        for (int q = 0; q < RT / 32; ++q) {
            const int32_t c = wcnt[q][threadIdx.x];
            wcnt[q][threadIdx.x] = s;
            s += c;
        }
        base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RITEMS; ++r) {
        if (dgt[r] < 256u) {
            const int64_t pos = (int64_t)base[dgt[r]] + wcnt[w][dgt[r]] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

__global__ void gather_i32_kernel(const int32_t *src, const int32_t *ord, int64_t n, int32_t *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[ord[i]];
}

__global__ void gather_f32_kernel(const float *src, const int32_t *ord, int64_t n, float *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[ord[i]];
}

struct IdxPtrs {
    const int32_t *p[SPT_MAX_ORDER];
};

// Packed records of the mode-n sorted copy: rec[i] = {rows_sorted[i],
// idx[m][perm[i]] for m != n in increasing m, bits(vals[perm[i]]), 0 pad}.
__global__ void pack_records_kernel(IdxPtrs idx, int d, int n, const float *vals, const int32_t *perm,
                                    const int32_t *srows, int64_t P, int rw, int32_t *rec) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = perm[i];
        int32_t *r = rec + i * rw;
        r[0] = srows[i];
        int k = 1;
        for (int m = 0; m < d; ++m)
            if (m != n) r[k++] = idx.p[m][q];
        r[k++] = __float_as_int(vals[q]);
        for (; k < rw; ++k) r[k] = 0;
    }
}
struct IdxOut {
    int32_t *p[SPT_MAX_ORDER];
};

__global__ void head_flags_kernel(IdxPtrs idx, int d, const int32_t *ord, int64_t n, int32_t *head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int h = (i == 0);
        if (!h) {
            const int32_t a = ord[i], b = ord[i - 1];
            for (int m = 0; m < d; ++m)
                if (idx.p[m][a] != idx.p[m][b]) { h = 1; break; }
        }
        head[i] = h;
    }
}

__global__ void coalesce_scatter_kernel(IdxPtrs idx, int d, const float *vals, const int32_t *ord,
                                        const int32_t *head, const int32_t *pos, int64_t n,
                                        IdxOut nidx, double *dsum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = ord[i];
        const int32_t seg = pos[i] + head[i] - 1;
        if (head[i])
            for (int m = 0; m < d; ++m) nidx.p[m][seg] = idx.p[m][q];
        atomicAdd(dsum + seg, (double)vals[q]);
    }
}

__global__ void finish_vals_kernel(const double *dsum, int64_t n, float *vals, double *norm2) {
    double local = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)dsum[i];
        vals[i] = v;
        local += (double)v * (double)v;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(FULL, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(norm2, local);
}

__global__ void norm2_kernel(const float *vals, int64_t n, double *norm2) {
    double local = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        local += (double)vals[i] * (double)vals[i];
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(FULL, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(norm2, local);
}

// slice counts from the sorted mode-n coordinates (equal rows are adjacent,
// so one warp-aggregated atomic covers each run inside a warp)
__global__ void slice_count_kernel(const int32_t *rows, int64_t n, int32_t *cnt) {
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const int lane = threadIdx.x & 31;
        const bool valid = i < n;
        const int32_t r = valid ? rows[i] : -1;
        const unsigned peers = __match_any_sync(FULL, r);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(cnt + r, __popc(peers));
    }
}

struct StatAcc {
    unsigned long long nonempty;
    unsigned long long maxc;
    double sumsq;
    unsigned long long runs;
};

__global__ void slice_stats_kernel(const int32_t *cnt, int64_t I, StatAcc *acc) {
    unsigned long long ne = 0, mx = 0;
    double sq = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = (unsigned long long)cnt[i];
        ne += (c > 0);
        mx = c > mx ? c : mx;
        sq += (double)c * (double)c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ne += __shfl_xor_sync(FULL, ne, o);
        const unsigned long long y = __shfl_xor_sync(FULL, mx, o);
        mx = y > mx ? y : mx;
        sq += __shfl_xor_sync(FULL, sq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc->nonempty, ne);
        atomicMax(&acc->maxc, mx);
        atomicAdd(&acc->sumsq, sq);
    }
}

__global__ void storage_runs_kernel(const int32_t *rows, int64_t n, StatAcc *acc) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        c += (i == 0) || (rows[i] != rows[i - 1]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc->runs, c);
}

int grid_for(int64_t n, int threads) {
    const int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 8;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

int bit_width_u32(uint64_t x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}
}  // namespace

// ---- device memory helpers (stream-ordered) ----------------------------------
spt_status dmalloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SPT_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                    " bytes failed: " + cudaGetErrorString(e));
    }
    return SPT_OK;
}

void dfree(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// Exclusive prefix sum of n int32 (in-place allowed).  *total_dev (device,
// nullable) receives the sum of all n inputs.
spt_status scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev,
                          cudaStream_t st) {
    if (n <= 0) {
        if (total_dev) SPT_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int32_t), st));
        return SPT_OK;
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *sums = nullptr;
    spt_status s = dmalloc((void **)&sums, sizeof(int32_t) * nb, st);
    if (s) return s;
    scan_block_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, n, sums);
    SPT_LAUNCH_CHECK("scan_block_kernel");
    if (nb == 1) {
        if (total_dev) SPT_CUDA(cudaMemcpyAsync(total_dev, sums, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    } else {
        s = scan_exclusive(sums, sums, nb, total_dev, st);
        if (s) { dfree(sums, st); return s; }
        scan_add_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(out, n, sums);
        SPT_LAUNCH_CHECK("scan_add_kernel");
    }
    dfree(sums, st);
    return SPT_OK;
}

// Stable sort of (key, value) pairs by the low `bits` bits of key.
// vals_in == nullptr means values 0..n-1 (the positions).
spt_status radix_sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, int64_t n, int bits,
                            uint32_t *keys_out, int32_t *vals_out, cudaStream_t st) {
    if (n <= 0) return SPT_OK;
    const int passes = std::max(1, (bits + 7) / 8);
    const int64_t ntiles = (n + RTILE - 1) / RTILE;
    int32_t *hist = nullptr;
    uint32_t *kb[2] = {nullptr, nullptr};
    int32_t *vb[2] = {nullptr, nullptr};
    spt_status s = dmalloc((void **)&hist, sizeof(int32_t) * 256 * ntiles, st);
    for (int q = 0; q < 2 && s == SPT_OK && passes > 1; ++q) {
        if (q == 1 && passes == 2) break;  // two passes need one intermediate buffer
        s = dmalloc((void **)&kb[q], sizeof(uint32_t) * n, st);
        if (!s) s = dmalloc((void **)&vb[q], sizeof(int32_t) * n, st);
    }
    for (int p = 0; p < passes && s == SPT_OK; ++p) {
        const uint32_t *ik = p == 0 ? keys_in : kb[(p - 1) & 1];
        const int32_t *iv = p == 0 ? vals_in : vb[(p - 1) & 1];
        uint32_t *ok = p == passes - 1 ? keys_out : kb[p & 1];
        int32_t *ov = p == passes - 1 ? vals_out : vb[p & 1];
        radix_hist_kernel<<<(unsigned)ntiles, RT, 0, st>>>(ik, n, 8 * p, hist, ntiles);
        if (cudaGetLastError() != cudaSuccess) { s = fail(SPT_ECUDA, "radix_hist_kernel launch"); break; }
        s = scan_exclusive(hist, hist, 256 * ntiles, nullptr, st);
        if (s) break;
        radix_scatter_kernel<<<(unsigned)ntiles, RT, 0, st>>>(ik, iv, n, 8 * p, hist, ntiles, ok, ov);
        if (cudaGetLastError() != cudaSuccess) { s = fail(SPT_ECUDA, "radix_scatter_kernel launch"); break; }
    }
    dfree(hist, st);
    for (int q = 0; q < 2; ++q) { dfree(kb[q], st); dfree(vb[q], st); }
    return s;
}

// Sum duplicate coordinates: lexicographic LSD sort over modes d-1..0, head
// flags, compaction, FP64 sums (rounded once to float32), and ||X||^2.
spt_status coalesce_tensor(spt_tensor t, cudaStream_t st) {
    const int64_t n = t->nnz;
    const int d = t->d;
    if (n == 0) { t->coalesced = true; t->xnorm2 = 0.0; return SPT_OK; }
    int32_t *ord = nullptr, *ord2 = nullptr, *head = nullptr, *pos = nullptr, *ucount = nullptr;
    uint32_t *k1 = nullptr, *k2 = nullptr;
    double *dsum = nullptr, *dnorm = nullptr;
    void *nbuf = nullptr;
    spt_status s = SPT_OK;
    auto cleanup = [&]() {
        dfree(ord, st); dfree(ord2, st); dfree(head, st); dfree(pos, st); dfree(ucount, st);
        dfree(k1, st); dfree(k2, st); dfree(dsum, st); dfree(dnorm, st);
    };
    s = dmalloc((void **)&ord, 4 * n, st);
    if (!s) s = dmalloc((void **)&ord2, 4 * n, st);
    if (!s) s = dmalloc((void **)&k1, 4 * n, st);
    if (!s) s = dmalloc((void **)&k2, 4 * n, st);
    if (s) { cleanup(); return s; }
    const int g = grid_for(n, 256);
    for (int m = d - 1; m >= 0 && !s; --m) {
        const int bits = bit_width_u32((uint64_t)(t->dims[m] - 1));
        if (m == d - 1) {
            s = radix_sort_pairs(reinterpret_cast<const uint32_t *>(t->idx[m]), nullptr, n, bits, k2, ord, st);
        } else {
            gather_i32_kernel<<<g, 256, 0, st>>>(t->idx[m], ord, n, reinterpret_cast<int32_t *>(k1));
            s = radix_sort_pairs(k1, ord, n, bits, k2, ord2, st);
            std::swap(ord, ord2);
        }
    }
    if (!s) s = dmalloc((void **)&head, 4 * n, st);
    if (!s) s = dmalloc((void **)&pos, 4 * n, st);
    if (!s) s = dmalloc((void **)&ucount, 4, st);
    if (s) { cleanup(); return s; }
    IdxPtrs ip;
    for (int m = 0; m < d; ++m) ip.p[m] = t->idx[m];
    head_flags_kernel<<<g, 256, 0, st>>>(ip, d, ord, n, head);
    SPT_LAUNCH_CHECK("head_flags_kernel");
    s = scan_exclusive(head, pos, n, ucount, st);
    if (s) { cleanup(); return s; }
    int32_t U = 0;
    SPT_CUDA(cudaMemcpyAsync(&U, ucount, 4, cudaMemcpyDeviceToHost, st));
    SPT_CUDA(cudaStreamSynchronize(st));
    const size_t seg = seg_bytes(U, 4);
    s = dmalloc(&nbuf, seg * (d + 1), st);
    if (!s) s = dmalloc((void **)&dsum, sizeof(double) * std::max<int64_t>(U, 1), st);
    if (!s) s = dmalloc((void **)&dnorm, sizeof(double), st);
    if (s) { dfree(nbuf, st); cleanup(); return s; }
    IdxOut no;
    for (int m = 0; m < d; ++m) no.p[m] = reinterpret_cast<int32_t *>((char *)nbuf + seg * m);
    float *nvals = reinterpret_cast<float *>((char *)nbuf + seg * d);
    SPT_CUDA(cudaMemsetAsync(dsum, 0, sizeof(double) * std::max<int64_t>(U, 1), st));
    SPT_CUDA(cudaMemsetAsync(dnorm, 0, sizeof(double), st));
    coalesce_scatter_kernel<<<g, 256, 0, st>>>(ip, d, t->vals, ord, head, pos, n, no, dsum);
    SPT_LAUNCH_CHECK("coalesce_scatter_kernel");
    finish_vals_kernel<<<grid_for(U, 256), 256, 0, st>>>(dsum, U, nvals, dnorm);
    SPT_LAUNCH_CHECK("finish_vals_kernel");
    double x2 = 0.0;
    SPT_CUDA(cudaMemcpyAsync(&x2, dnorm, sizeof(double), cudaMemcpyDeviceToHost, st));
    cleanup();
    SPT_CUDA(cudaStreamSynchronize(st));
    dfree(t->coo_buf, st);
    t->coo_buf = nbuf;
    for (int m = 0; m < d; ++m) t->idx[m] = no.p[m];
    t->vals = nvals;
    t->nnz = U;
    t->coalesced = true;
    t->xnorm2 = x2;
    return SPT_OK;
}

// Permutation of mode n (and the mode-sorted copy unless index_only), plus
// slice statistics.  Synchronises `st` at the end.
spt_status build_perm_mode(spt_tensor t, int n, bool index_only, cudaStream_t st, bool slice_order) {
    const int64_t P = t->nnz;
    const int d = t->d;
    // release an earlier build of this mode
    if (t->perm[n]) { cudaFreeAsync(t->perm[n], st); t->perm[n] = nullptr; }
    if (t->sorted_buf[n]) { cudaFreeAsync(t->sorted_buf[n], st); t->sorted_buf[n] = nullptr; }
    if (t->blk_buf[n]) { cudaFreeAsync(t->blk_buf[n], st); t->blk_buf[n] = nullptr; }  // built from the old copy
    t->blk_off[n].clear();
    t->blk_mode[n] = -1;
    t->blk_rows[n] = 0;
    int32_t *perm = nullptr, *srows = nullptr;
    spt_status s = dmalloc((void **)&perm, seg_bytes(P, 4), st);
    if (!s) s = dmalloc((void **)&srows, seg_bytes(P, 4), st);
    if (s) { dfree(perm, st); return s; }
    const int bits = bit_width_u32((uint64_t)(t->dims[n] - 1));
    s = radix_sort_pairs(reinterpret_cast<const uint32_t *>(t->idx[n]), nullptr, P, bits,
                         reinterpret_cast<uint32_t *>(srows), perm, st);
    if (s) { dfree(perm, st); dfree(srows, st); return s; }
    const int g = grid_for(P, 256);
    if (!index_only) {
        // The copy's order: perm_n, or with slice_order by mode n and inside
        // a slice by the next modes (n+1, then n+2, cyclically; ties in
        // storage order), so that neighbouring nonzeros of a long slice
        // repeat factor rows.  A stable LSD sort: mode n+2, then mode n+1,
        // then mode n.
        int32_t *ord = nullptr, *ord2 = nullptr;
        uint32_t *kin = nullptr, *kout = nullptr;
        const int nsec = slice_order ? std::min(2, d - 1) : 0;
        if (nsec > 0 && P > 0) {
            s = dmalloc((void **)&ord, seg_bytes(P, 4), st);
            if (!s) s = dmalloc((void **)&ord2, seg_bytes(P, 4), st);
            if (!s) s = dmalloc((void **)&kin, seg_bytes(P, 4), st);
            if (!s) s = dmalloc((void **)&kout, seg_bytes(P, 4), st);
            for (int q = nsec; q >= 0 && !s; --q) {
                const int m = (n + q) % d;
                const int mb = bit_width_u32((uint64_t)(t->dims[m] - 1));
                if (q == nsec) {
                    s = radix_sort_pairs(reinterpret_cast<const uint32_t *>(t->idx[m]), nullptr, P, mb, kout, ord,
                                         st);
                } else {
                    gather_i32_kernel<<<g, 256, 0, st>>>(t->idx[m], ord, P, reinterpret_cast<int32_t *>(kin));
                    s = radix_sort_pairs(kin, ord, P, mb, kout, ord2, st);
                    std::swap(ord, ord2);
                }
            }
        }
        const int rw = record_words(d);
        void *sbuf = nullptr;
        if (!s) s = dmalloc(&sbuf, seg_bytes(P * rw, 4), st);
        if (s) {
            dfree(ord, st); dfree(ord2, st); dfree(kin, st); dfree(kout, st);
            dfree(perm, st); dfree(srows, st);
            return s;
        }
        IdxPtrs ip;
        for (int m = 0; m < d; ++m) ip.p[m] = t->idx[m];
        if (P > 0)  // the copy's mode-n keys equal srows: both orders sort by mode n first
            pack_records_kernel<<<g, 256, 0, st>>>(ip, d, n, t->vals, ord ? ord : perm, srows, P, rw,
                                                   reinterpret_cast<int32_t *>(sbuf));
        SPT_LAUNCH_CHECK("pack_records_kernel");
        dfree(ord, st); dfree(ord2, st); dfree(kin, st); dfree(kout, st);
        t->sorted_buf[n] = sbuf;
    }
    t->perm[n] = perm;
    // slice statistics
    int32_t *cnt = nullptr;
    StatAcc *acc = nullptr;
    s = dmalloc((void **)&cnt, 4 * t->dims[n], st);
    if (!s) s = dmalloc((void **)&acc, sizeof(StatAcc), st);
    if (s) { dfree(srows, st); dfree(cnt, st); return s; }
    SPT_CUDA(cudaMemsetAsync(cnt, 0, 4 * t->dims[n], st));
    SPT_CUDA(cudaMemsetAsync(acc, 0, sizeof(StatAcc), st));
    if (P > 0) {
        slice_count_kernel<<<g, 256, 0, st>>>(srows, P, cnt);
        storage_runs_kernel<<<g, 256, 0, st>>>(t->idx[n], P, acc);
    }
    slice_stats_kernel<<<grid_for(t->dims[n], 256), 256, 0, st>>>(cnt, t->dims[n], acc);
    SPT_LAUNCH_CHECK("slice statistics kernels");
    StatAcc h{};
    SPT_CUDA(cudaMemcpyAsync(&h, acc, sizeof(StatAcc), cudaMemcpyDeviceToHost, st));
    dfree(cnt, st);
    dfree(acc, st);
    dfree(srows, st);
    SPT_CUDA(cudaStreamSynchronize(st));
    ModeStats &ms = t->stats[n];
    ms.valid = true;
    ms.nonempty = (int64_t)h.nonempty;
    ms.max_count = (int64_t)h.maxc;
    ms.sum_sq = h.sumsq;
    ms.runs_storage = (int64_t)h.runs;
    return SPT_OK;
}

spt_status compute_norm2(spt_tensor t, cudaStream_t st) {
    double *dn = nullptr;
    spt_status s = dmalloc((void **)&dn, sizeof(double), st);
    if (s) return s;
    SPT_CUDA(cudaMemsetAsync(dn, 0, sizeof(double), st));
    if (t->nnz > 0) norm2_kernel<<<grid_for(t->nnz, 256), 256, 0, st>>>(t->vals, t->nnz, dn);
    SPT_LAUNCH_CHECK("norm2_kernel");
    double x2 = 0.0;
    SPT_CUDA(cudaMemcpyAsync(&x2, dn, sizeof(double), cudaMemcpyDeviceToHost, st));
    dfree(dn, st);
    SPT_CUDA(cudaStreamSynchronize(st));
    t->xnorm2 = x2;
    return SPT_OK;
}

namespace {
// flag[r] = 1 for rows with at least minc nonzeros
__global__ void hot_flag_kernel(const int32_t *cnt, int64_t I, int32_t minc, int32_t *flag) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = cnt[r] >= minc ? 1 : 0;
}

// s[0] += sum count^2, s[1] += sum count^3 over the rows
__global__ void count_moments_kernel(const int32_t *cnt, int64_t I, double *s) {
    double a = 0.0, b = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x) {
        const double c = (double)cnt[r];
        a += c * c;
        b += c * c * c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL, a, o);
        b += __shfl_xor_sync(FULL, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(s, a);
        atomicAdd(s + 1, b);
    }
}

// candidates in row order: key = P - count (so an ascending sort puts the
// hottest first), value = row
__global__ void hot_compact_kernel(const int32_t *cnt, const int32_t *flag, const int32_t *pos, int64_t I,
                                   uint32_t P, uint32_t *keys, int32_t *rows) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) {
            keys[pos[r]] = P - (uint32_t)cnt[r];
            rows[pos[r]] = (int32_t)r;
        }
}
}  // namespace

// Per mode: count each row's nonzeros, keep the rows with at least
// SPT_HOT_MIN_COUNT of them (in row order, by a flag scan), sort those by
// count (stable, so ties stay in row order) and record the first SPT_HOT_MAX.
// rec[i] = {idx[0][i], ..., idx[d-1][i], bits(vals[i]), 0 pad}
__global__ void storage_records_kernel(IdxPtrs idx, int d, const float *vals, int64_t P, int rw, int32_t *rec) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t *r = rec + i * rw;
        for (int m = 0; m < d; ++m) r[m] = idx.p[m][i];
        r[d] = __float_as_int(vals[i]);
        for (int k = d + 1; k < rw; ++k) r[k] = 0;
    }
}

spt_status build_storage_records(spt_tensor t, cudaStream_t st) {
    const int rw = record_words(t->d);
    int32_t *rec = nullptr;
    spt_status s = dmalloc((void **)&rec, seg_bytes(std::max<int64_t>(1, t->nnz) * rw, 4), st);
    if (s) return s;
    IdxPtrs ip;
    for (int m = 0; m < t->d; ++m) ip.p[m] = t->idx[m];
    if (t->nnz > 0)
        storage_records_kernel<<<grid_for(t->nnz, 256), 256, 0, st>>>(ip, t->d, t->vals, t->nnz, rw, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { dfree(rec, st); return cuda_fail(e, "build_storage_records"); }
    t->srec = rec;
    return SPT_OK;
}

// keys[i] = (word k of record i) / block_rows
__global__ void block_keys_kernel(const int32_t *rec, int rw, int k, int64_t P, int64_t block_rows, uint32_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)(rec[i * rw + k] / block_rows);
}

// record order[i] of src -> dst position i + shift[key[i]] (the stable order
// by block puts each block's records at its padded offset)
__global__ void block_scatter_kernel(const int32_t *src, int rw, const int32_t *order, const uint32_t *skeys,
                                     const int64_t *shift, int64_t P, int32_t *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *a = src + (int64_t)order[i] * rw;
        int32_t *b = dst + (i + shift[skeys[i]]) * rw;
        for (int w = 0; w < rw; ++w) b[w] = a[w];
    }
}

// pad slot j of block b: a copy of the block's last record with value 0
__global__ void block_pad_kernel(const int64_t *pad_at, const int64_t *pad_src, int64_t npad, int rw, int vword,
                                 int32_t *dst) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < npad; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *a = dst + pad_src[j] * rw;
        int32_t *b = dst + pad_at[j] * rw;
        for (int w = 0; w < rw; ++w) b[w] = w == vword ? 0 : a[w];
    }
}

spt_status build_l2_blocks(spt_tensor t, int n, int bm, int64_t block_rows, cudaStream_t st) {
    const int64_t P = t->nnz;
    const int d = t->d;
    const int rw = record_words(d);
    if (t->blk_buf[n]) { cudaFreeAsync(t->blk_buf[n], st); t->blk_buf[n] = nullptr; }
    t->blk_off[n].clear();
    t->blk_mode[n] = -1;
    t->blk_rows[n] = 0;
    const int64_t nb = (t->dims[bm] + block_rows - 1) / block_rows;
    const int k = 1 + (bm < n ? bm : bm - 1);  // the record word of mode bm
    const int32_t *src = reinterpret_cast<const int32_t *>(t->sorted_buf[n]);
    uint32_t *keys = nullptr, *skeys = nullptr;
    int32_t *order = nullptr, *cnt = nullptr;
    int64_t *dshift = nullptr, *dpad = nullptr;
    void *buf = nullptr;
    auto cleanup = [&]() {
        dfree(keys, st); dfree(skeys, st); dfree(order, st); dfree(cnt, st); dfree(dshift, st); dfree(dpad, st);
    };
    spt_status s = dmalloc((void **)&keys, seg_bytes(P, 4), st);
    if (!s) s = dmalloc((void **)&skeys, seg_bytes(P, 4), st);
    if (!s) s = dmalloc((void **)&order, seg_bytes(P, 4), st);
    if (!s) s = dmalloc((void **)&cnt, 4 * nb, st);
    if (s) { cleanup(); return s; }
    SPT_CUDA(cudaMemsetAsync(cnt, 0, 4 * nb, st));
    std::vector<int32_t> hcnt(nb, 0);
    if (P > 0) {
        block_keys_kernel<<<grid_for(P, 256), 256, 0, st>>>(src, rw, k, P, block_rows, keys);
        s = radix_sort_pairs(keys, nullptr, P, bit_width_u32((uint64_t)(nb - 1)), skeys, order, st);
        if (s) { cleanup(); return s; }
        slice_count_kernel<<<grid_for(P, 256), 256, 0, st>>>(reinterpret_cast<const int32_t *>(skeys), P, cnt);
        SPT_LAUNCH_CHECK("block key kernels");
        cudaError_t e = cudaMemcpyAsync(hcnt.data(), cnt, 4 * nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "build_l2_blocks counts"); }
    }
    // padded offsets (multiples of 4 records keep every group 16-byte aligned)
    std::vector<int64_t> off(nb + 1, 0), shift(nb, 0), pad_at, pad_src;
    int64_t start = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t c = hcnt[b], pc = (c + 3) & ~int64_t(3);
        off[b + 1] = off[b] + pc;
        shift[b] = off[b] - start;
        for (int64_t j = c; j < pc; ++j) {
            pad_at.push_back(off[b] + j);
            pad_src.push_back(off[b] + c - 1);
        }
        start += c;
    }
    const int64_t npad = (int64_t)pad_at.size();
    s = dmalloc(&buf, seg_bytes(std::max<int64_t>(1, off[nb]) * rw, 4), st);
    if (!s) s = dmalloc((void **)&dshift, sizeof(int64_t) * std::max<int64_t>(1, nb), st);
    if (!s) s = dmalloc((void **)&dpad, sizeof(int64_t) * std::max<int64_t>(1, 2 * npad), st);
    if (s) { cleanup(); dfree(buf, st); return s; }
    std::vector<int64_t> hpad(pad_at);
    hpad.insert(hpad.end(), pad_src.begin(), pad_src.end());
    cudaError_t e = cudaMemcpyAsync(dshift, shift.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && npad > 0)
        e = cudaMemcpyAsync(dpad, hpad.data(), sizeof(int64_t) * 2 * npad, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { cleanup(); dfree(buf, st); return cuda_fail(e, "build_l2_blocks tables"); }
    if (P > 0)
        block_scatter_kernel<<<grid_for(P, 256), 256, 0, st>>>(src, rw, order, skeys, dshift, P,
                                                               reinterpret_cast<int32_t *>(buf));
    if (npad > 0)
        block_pad_kernel<<<grid_for(npad, 256), 256, 0, st>>>(dpad, dpad + npad, npad, rw, d,
                                                              reinterpret_cast<int32_t *>(buf));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables go out of scope
    cleanup();
    if (e != cudaSuccess) { dfree(buf, st); return cuda_fail(e, "build_l2_blocks copy"); }
    t->blk_buf[n] = buf;
    t->blk_off[n] = off;
    t->blk_mode[n] = bm;
    t->blk_rows[n] = block_rows;
    return SPT_OK;
}

spt_status build_hot_rows(spt_tensor t, cudaStream_t st) {
    const int64_t P = t->nnz;
    if (!t->hot_buf) {
        spt_status s = dmalloc((void **)&t->hot_buf, sizeof(int32_t) * SPT_HOT_MAX * SPT_MAX_ORDER, st);
        if (s) return s;
    }
    for (int n = 0; n < t->d; ++n) {
        t->nhot[n] = 0;
        for (int k = 0; k <= SPT_HOT_MAX; ++k) t->hot_count[n][k] = 0;
        t->cnt_s2[n] = t->cnt_s3[n] = 0.0;
    }
    if (P < SPT_HOT_MIN_COUNT) return SPT_OK;
    for (int n = 0; n < t->d; ++n) {
        const int64_t I = t->dims[n];
        int32_t *cnt = nullptr, *flag = nullptr, *pos = nullptr, *total = nullptr, *rows = nullptr, *srows = nullptr;
        uint32_t *keys = nullptr, *skeys = nullptr;
        double *mom = nullptr;
        auto cleanup = [&]() {
            dfree(cnt, st); dfree(flag, st); dfree(pos, st); dfree(total, st);
            dfree(rows, st); dfree(srows, st); dfree(keys, st); dfree(skeys, st); dfree(mom, st);
        };
        spt_status s = dmalloc((void **)&cnt, 4 * I, st);
        if (!s) s = dmalloc((void **)&flag, 4 * I, st);
        if (!s) s = dmalloc((void **)&pos, 4 * I, st);
        if (!s) s = dmalloc((void **)&total, 4, st);
        if (!s) s = dmalloc((void **)&mom, 2 * sizeof(double), st);
        if (s) { cleanup(); return s; }
        cudaError_t e = cudaMemsetAsync(cnt, 0, 4 * I, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(mom, 0, 2 * sizeof(double), st);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "build_hot_rows memset"); }
        slice_count_kernel<<<grid_for(P, 256), 256, 0, st>>>(t->idx[n], P, cnt);
        hot_flag_kernel<<<grid_for(I, 256), 256, 0, st>>>(cnt, I, SPT_HOT_MIN_COUNT, flag);
        count_moments_kernel<<<grid_for(I, 256), 256, 0, st>>>(cnt, I, mom);
        e = cudaGetLastError();
        if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "build_hot_rows kernels"); }
        s = scan_exclusive(flag, pos, I, total, st);
        int32_t nc = 0;
        double hm[2] = {0.0, 0.0};
        if (!s) {
            e = cudaMemcpyAsync(&nc, total, 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hm, mom, sizeof(hm), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(e, "build_hot_rows count");
        }
        t->cnt_s2[n] = hm[0];
        t->cnt_s3[n] = hm[1];
        if (!s && nc > 0) {
            s = dmalloc((void **)&keys, 4 * (size_t)nc, st);
            if (!s) s = dmalloc((void **)&rows, 4 * (size_t)nc, st);
            if (!s) s = dmalloc((void **)&skeys, 4 * (size_t)nc, st);
            if (!s) s = dmalloc((void **)&srows, 4 * (size_t)nc, st);
            if (!s) {
                hot_compact_kernel<<<grid_for(I, 256), 256, 0, st>>>(cnt, flag, pos, I, (uint32_t)P, keys, rows);
                e = cudaGetLastError();
                if (e != cudaSuccess) s = cuda_fail(e, "hot_compact_kernel");
            }
            if (!s) s = radix_sort_pairs(keys, rows, nc, bit_width_u32((uint64_t)P), skeys, srows, st);
            const int k = std::min<int32_t>(nc, SPT_HOT_MAX);
            uint32_t hk[SPT_HOT_MAX + 1];
            const int kc = std::min<int32_t>(nc, SPT_HOT_MAX + 1);
            if (!s) {
                e = cudaMemcpyAsync(t->hot_buf + (size_t)n * SPT_HOT_MAX, srows, 4 * (size_t)k,
                                    cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(hk, skeys, 4 * (size_t)kc, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) s = cuda_fail(e, "build_hot_rows copy");
            }
            if (!s) {
                t->nhot[n] = k;
                for (int q = 0; q < kc; ++q) t->hot_count[n][q] = (int64_t)P - (int64_t)hk[q];
            }
        }
        cleanup();
        if (s) return s;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? SPT_OK : cuda_fail(e, "build_hot_rows");
}

// ---------------------------------------------------------------------------
// Allocation-free mode permutation.
//
// Some callers cannot allocate device memory when they need a permutation:
// code running inside someone else's fixed memory budget (a serving process
// whose pool owns every byte of the GPU), code that must not trigger the
// device-wide synchronisation cudaFree implies, or a driver that sets up all
// memory once and then only launches work.  For them this entry point sorts
// with a scratch area that is part of the library image itself: a static
// device array, created when the library is loaded on a GPU and kept until
// the process exits.  The caller passes the coordinates in and receives the
// permutation; nothing is allocated or freed on the way.
//
// The area holds the two ping-pong key/position buffers of the radix sort,
// the digit histogram and the scan's block sums, which bounds n to
// SPT_NOALLOC_MAX_NNZ.  Every pass overwrites what the next one reads, so
// nothing in the area has to start at zero.  All calls in the process share
// the one area: calls whose work overlaps on the GPU (other streams, other
// host threads) race on it and must be ordered by the caller.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB per GPU
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch area on the current device.  In host code
// the array's name is only a host-side stand-in, so every call asks the
// runtime for the address with the caller's device current (no allocation,
// and never a stale address after a device reset re-creates the context).
// The first lookup on a device also loads the library's device code there.
spt_status noalloc_scratch(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    *out = p;
    return SPT_OK;
}

struct Carve {
    char *p;
    size_t left;
    template <typename T> T *take(size_t count) {
        const size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
        if (bytes > left) return nullptr;
        T *r = reinterpret_cast<T *>(p);
        p += bytes;
        left -= bytes;
        return r;
    }
};

// In-place exclusive scan with block sums carved from the static area.
spt_status scan_inplace_carved(int32_t *data, int64_t n, Carve &cv, cudaStream_t st) {
    if (n <= 0) return SPT_OK;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *sums = cv.take<int32_t>(nb);
    if (!sums) return fail(SPT_EINVAL, "noalloc scratch exhausted in scan");
    scan_block_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(data, data, n, sums);
    SPT_LAUNCH_CHECK("scan_block_kernel");
    if (nb > 1) {
        spt_status s = scan_inplace_carved(sums, nb, cv, st);
        if (s) return s;
        scan_add_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(data, n, sums);
        SPT_LAUNCH_CHECK("scan_add_kernel");
    }
    return SPT_OK;
}
}  // namespace

}  // namespace spt

using namespace spt;

extern "C" spt_status mode_permutation_noalloc(const int32_t *keys, int64_t n, int64_t dim,
                                               int32_t *perm, void *stream) {
    if (n < 0 || n > SPT_NOALLOC_MAX_NNZ)
        return fail(SPT_EINVAL, "mode_permutation_noalloc: n must be in [0, " +
                                    std::to_string((long long)SPT_NOALLOC_MAX_NNZ) +
                                    "] (the size of the static scratch area)");
    if (dim < 1 || dim > INT32_MAX) return fail(SPT_EINVAL, "mode_permutation_noalloc: dim must be in [1, 2^31-1]");
    if (n == 0) return SPT_OK;
    if (!keys || !perm) return fail(SPT_EINVAL, "mode_permutation_noalloc: NULL keys or perm");
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    spt_status s = noalloc_scratch(&base);
    if (s) return s;
    Carve cv{reinterpret_cast<char *>(base), NOALLOC_SCRATCH_BYTES};
    const int bits = bit_width_u32((uint64_t)(dim - 1));
    const int passes = std::max(1, (bits + 7) / 8);
    const int64_t ntiles = (n + RTILE - 1) / RTILE;
    uint32_t *kb[2] = {cv.take<uint32_t>(n), cv.take<uint32_t>(n)};
    int32_t *vb[2] = {cv.take<int32_t>(n), cv.take<int32_t>(n)};
    int32_t *hist = cv.take<int32_t>(256 * ntiles);
    if (!kb[0] || !kb[1] || !vb[0] || !vb[1] || !hist)
        return fail(SPT_EINVAL, "mode_permutation_noalloc: n too large for the static scratch area");
    for (int p = 0; p < passes; ++p) {
        const uint32_t *ik = p == 0 ? reinterpret_cast<const uint32_t *>(keys) : kb[(p - 1) & 1];
        const int32_t *iv = p == 0 ? nullptr : vb[(p - 1) & 1];
        int32_t *ov = p == passes - 1 ? perm : vb[p & 1];
        radix_hist_kernel<<<(unsigned)ntiles, RT, 0, st>>>(ik, n, 8 * p, hist, ntiles);
        SPT_LAUNCH_CHECK("radix_hist_kernel");
        Carve scan_cv = cv;  // the scan's block sums reuse the same tail every pass
        s = scan_inplace_carved(hist, 256 * ntiles, scan_cv, st);
        if (s) return s;
        radix_scatter_kernel<<<(unsigned)ntiles, RT, 0, st>>>(ik, iv, n, 8 * p, hist, ntiles,
                                                             kb[p & 1], ov);
        SPT_LAUNCH_CHECK("radix_scatter_kernel");
    }
    return SPT_OK;
}

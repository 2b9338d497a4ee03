// cpals.cu -- one CP-ALS iteration on the device (Sec. 3: alternating least
// squares; the MTTKRP of Sec. 3 eq. mttkrp is its dominant step).
//
// Per mode n (in order 0..d-1):
//   1. V = MTTKRP_n(X, A)                                (mttkrp kernel)
//   2. H = *_{m != n} G_m, Hinv = H^-1 by symmetric Gauss-Jordan
//      elimination, whose pivots are the squared diagonal of H's
//      Cholesky factor                                    (one CTA, FP64)
//   3. A32 = V Hinv, colsq_j = sum_k A32(k,j)^2           (FP32 FMAs, FP64 sums)
//   4. lambda_j = sqrt(colsq_j), A^(n) = A32 / lambda   -> stored type
//      (round to nearest even for 16-bit factors)
//   5. G_n = A^(n)T A^(n) of the stored values           (FP32 partials over
//      row tiles, accumulated in FP64)
// After the last mode: fit = 1 - sqrt(max(0, ||X||^2 + ||M||^2 - 2<X,M>))/||X||
// with ||M||^2 = lambda^T (*_m G_m) lambda and <X,M> = sum V(k,j) lambda_j
// A^(d)(k,j) over the last mode's V.
//
// GB300 has little FP64 throughput, so FP64 is kept to the R x R work and to
// reductions; every O(I R^2) loop runs FP32 FMAs with FP64 accumulation of
// short partial sums.
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace spt {
namespace {

constexpr int MAXR = 128;
constexpr unsigned FULL = 0xffffffffu;

template <typename FT> __device__ __forceinline__ float ld_elem(const FT *p);
template <> __device__ __forceinline__ float ld_elem<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ld_elem<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float ld_elem<__half>(const __half *p) { return __half2float(*p); }

template <typename FT> __device__ __forceinline__ FT st_elem(float v);
template <> __device__ __forceinline__ float st_elem<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_elem<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half st_elem<__half>(float v) { return __float2half_rn(v); }

// 16-byte asynchronous copy global -> shared (cp.async, L1-allocating);
// src_bytes = 0 writes zeros without reading src.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Four consecutive stored elements widened to float.
template <typename FT> __device__ __forceinline__ float4 quad_f(const FT *p);
template <> __device__ __forceinline__ float4 quad_f<float>(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}
template <> __device__ __forceinline__ float4 quad_f<__nv_bfloat16>(const __nv_bfloat16 *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
template <> __device__ __forceinline__ float4 quad_f<__half>(const __half *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Shape of the Gram kernel for rank R and element size es: threads, rows of
// a tile per team (at most 16), tile rows, shared-memory row stride
// (elements) and bytes.
struct GramShape {
    int threads, rows_per_team, tile_rows, stride;
    size_t smem;
};
__host__ __device__ inline GramShape gram_shape(int R, int es) {
    const int RT = (R + 3) / 4, RP = 4 * RT, team = RT * RT;
    const int qb = 16 / es;  // elements per 16-byte piece
    GramShape g;
    g.threads = team >= 256 ? team : (256 / team) * team;
    const int RS = g.threads / team;
    g.stride = (RP + qb - 1) / qb * qb + qb;
    int rpt = 16;
    while (rpt > 1 && (size_t)2 * RS * rpt * g.stride * es > 48 * 1024) --rpt;
    g.rows_per_team = rpt;
    g.tile_rows = RS * rpt;
    g.smem = (size_t)2 * g.tile_rows * g.stride * es + sizeof(double) * (size_t)RS * RP * RP;
    return g;
}

// At most this many CTAs per SM run a Gram launch (and so the two-stage
// reduction holds at most SMs times this many partial Grams).
inline int gram_ctas_per_sm(int R) { return std::max(1, 1024 / gram_shape(R, 4).threads); }

// G += A^T A over all I rows (A row-major, stride ld, first R columns).
// Thread (ti, tj) of a team owns the 4 x 4 block G[4ti.., 4tj..] in
// registers; the RS teams of a CTA split the rows of each tile.  Tiles of
// raw stored rows are double buffered with cp.async, so the next tile loads
// while this one is multiplied.  Entries of G outside R x R (from padding
// columns, whatever they hold) are dropped at the end.  FP32 partial sums
// over at most 256 rows are folded into the team's FP64 copy of G in shared
// memory (one writer per entry); at the end the CTA sums its teams' copies
// in team order and either stores the sum as its R x R block of `partials`
// (row blockIdx.x; gram_reduce_kernel adds the blocks to G in block order)
// or, with partials = NULL, adds it to G atomically.
template <typename FT>
__global__ void __launch_bounds__(1024) gram_kernel(const FT *A, int64_t I, int ld, int R, double *G,
                                                    double *partials) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const GramShape sh = gram_shape(R, (int)sizeof(FT));
    const int RT = (R + 3) / 4, RP = RT * 4;
    const int team_sz = RT * RT;
    const int RS = blockDim.x / team_sz;
    const int TR = sh.tile_rows, SPE = sh.stride;
    constexpr int QB = 16 / (int)sizeof(FT);
    const int PR = (RP + QB - 1) / QB;  // 16-byte pieces per row (within ld)
    FT *const tile0 = reinterpret_cast<FT *>(gsm);  // two tiles of TR x SPE
    const size_t tsz = (size_t)TR * SPE;
    double *red = reinterpret_cast<double *>(gsm + (size_t)2 * TR * SPE * sizeof(FT));
    const int team = threadIdx.x / team_sz, tid = threadIdx.x % team_sz;
    const int ti = tid / RT, tj = tid % RT;
    const int RR = RP * RP;
    for (int e = threadIdx.x; e < RS * RR; e += blockDim.x) red[e] = 0.0;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    // fold the FP32 partials into the team's FP64 block (a thread: its entries)
    auto fold = [&]() {
        if (team < RS) {
            double *tred = red + (size_t)team * RR;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    tred[(4 * ti + i) * RP + 4 * tj + j] += (double)acc[i][j];
                    acc[i][j] = 0.f;
                }
        }
    };
    auto issue = [&](int64_t r0, FT *buf) {
        for (int e = threadIdx.x; e < TR * PR; e += blockDim.x) {
            const int r = e / PR, q = e - r * PR;
            const bool in = r0 + r < I;
            cp_async16(buf + (size_t)r * SPE + q * QB, in ? (const void *)(A + (r0 + r) * ld + q * QB) : A,
                       in ? 16 : 0);
        }
        cp_async_commit();
    };
    const int64_t step = (int64_t)gridDim.x * TR;
    int64_t r0 = (int64_t)blockIdx.x * TR;
    __syncthreads();  // red zeroed before the first fold
    if (r0 < I) issue(r0, tile0);
    int since = 0, k = 0;
    for (; r0 < I; r0 += step, ++k) {
        const bool next = r0 + step < I;
        if (next) issue(r0 + step, tile0 + ((k + 1) & 1) * tsz);
        if (next) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncthreads();
        const FT *buf = tile0 + (k & 1) * tsz;
        if (team < RS) {
            const int rmax = (int)(I - r0 < (int64_t)TR ? I - r0 : (int64_t)TR);
            for (int r = team; r < rmax; r += RS) {
                const float4 a = quad_f<FT>(buf + (size_t)r * SPE + 4 * ti);
                const float4 b = quad_f<FT>(buf + (size_t)r * SPE + 4 * tj);
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
        }
        since += sh.rows_per_team;
        if (since >= 256) {
            fold();
            since = 0;
        }
        __syncthreads();  // this buffer is refilled by the issue two tiles on
    }
    fold();
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        const int i = e / RP, j = e % RP;
        if (i >= R || j >= R) continue;
        double sum = 0.0;
        for (int t = 0; t < RS; ++t) sum += red[(size_t)t * RR + e];
        if (partials) partials[(int64_t)blockIdx.x * R * R + i * R + j] = sum;
        else atomicAdd(G + i * R + j, sum);
    }
}

// G += the sum of the nb partial Grams (R x R each, consecutive): a warp
// per entry, lane l adding blocks l, l + 32, ... (four loads in flight), the
// lanes' sums combined by a fixed shuffle tree, so the order of additions is
// fixed by nb alone.
__global__ void __launch_bounds__(256) gram_reduce_kernel(const double *partials, int nb, int RR, double *G) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= RR) return;  // warp-uniform
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int b = lane;
    for (; b + 96 < nb; b += 128) {
        s0 += partials[(int64_t)b * RR + e];
        s1 += partials[(int64_t)(b + 32) * RR + e];
        s2 += partials[(int64_t)(b + 64) * RR + e];
        s3 += partials[(int64_t)(b + 96) * RR + e];
    }
    for (; b < nb; b += 32) s0 += partials[(int64_t)b * RR + e];
    double sum = (s0 + s1) + (s2 + s3);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) G[e] += sum;
}

// H = *_{m != n} G_m and Hinv = H^-1 -> float, in FP64 with the sweep
// operator (Gauss-Jordan elimination kept symmetric; Goodnight, "A tutorial
// on the SWEEP operator", 1979): sweeping pivot k of a symmetric M with
// d = M(k,k) sets M(i,j) -= M(i,k) M(k,j) / d for i, j != k, M(i,k) =
// M(k,i) = M(i,k) / d, and M(k,k) = -1 / d; after every pivot M = -H^-1.
// Pivot k is the k-th diagonal entry of the Schur complement left by the
// earlier pivots -- the square L_kk^2 of H's Cholesky factor H = L L^T -- so
// the sweep runs to the end exactly when the Cholesky factorisation exists;
// a pivot <= 0 means H is not positive definite: one retry with a ridge of
// 1e-12 trace(H)/R, then the singular status and Hinv = identity.  M stays
// symmetric, so each step updates the R(R+1)/2 pairs i <= j with one FP64
// FMA each (GB300's FP64 rate is ~1/70 of its FP32 rate, so the FP64 work
// sets the time at larger R), all pairs at once: the critical path is 2R
// barriers, and the reciprocal of the next pivot is taken by the thread that
// updates it while the others update theirs.  The Cholesky-then-triangular-
// inverse form this replaces ran two R-long dependent chains on a few
// threads (27 us at R = 16, 233 us at R = 64 on GB300).  zero_gram / zero_colsq (nullable): R*R
// and R doubles cleared afterwards for this mode's update (G_n and the
// column sums).  Shared memory: R*R doubles (M), 2R doubles (column k and
// column k / d), R(R+1)/2 words (the pairs, i << 16 | j).
__global__ void __launch_bounds__(512) hinv_kernel(const double *G, int d, int n, int R, float *Hinv,
                                                   double *zero_gram, double *zero_colsq, int *status) {
    extern __shared__ double sh[];
    double *M = sh;           // R x R, symmetric
    double *ck = sh + R * R;  // R: column k before step k
    double *fk = ck + R;      // R: column k / pivot
    uint32_t *pairs = reinterpret_cast<uint32_t *>(fk + R);
    __shared__ double ridge, rpiv;  // rpiv: 1 / the next pivot (when it is > 0)
    const int RR = R * R, NP = R * (R + 1) / 2;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {  // the pairs, row by row
        const int i = e / R, j = e - i * R;
        if (j >= i) pairs[i * R - i * (i - 1) / 2 + (j - i)] = ((uint32_t)i << 16) | (uint32_t)j;
    }
    bool ok = false;
    for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
        __syncthreads();  // the pairs are written; the previous attempt's readers of M are done
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            double h = 1.0;
            for (int m = 0; m < d; ++m)
                if (m != n) h *= G[(int64_t)m * RR + e];
            M[e] = h;
        }
        __syncthreads();
        if (attempt == 1) {
            if (threadIdx.x == 0) {
                double tr = 0.0;
                for (int r = 0; r < R; ++r) tr += M[r * R + r];
                ridge = 1e-12 * tr / R;
            }
            __syncthreads();
            for (int r = threadIdx.x; r < R; r += blockDim.x) M[r * R + r] += ridge;
            __syncthreads();
        }
        ok = true;
        if (threadIdx.x == 0 && M[0] > 0.0) rpiv = 1.0 / M[0];
        __syncthreads();
        for (int k = 0; k < R; ++k) {
            const double piv = M[k * R + k];  // the same value in every thread
            if (!(piv > 0.0)) {
                ok = false;
                break;
            }
            const double rp = rpiv;
            for (int i = threadIdx.x; i < R; i += blockDim.x) {
                const double c = M[i * R + k];
                ck[i] = c;
                fk[i] = c * rp;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < NP; t += blockDim.x) {
                const uint32_t q = pairs[t];
                const int i = (int)(q >> 16), j = (int)(q & 0xffffu);
                double v;
                if (i == k && j == k) v = -rp;
                else if (i == k) v = fk[j];
                else if (j == k) v = fk[i];
                else v = fma(-fk[i], ck[j], M[i * R + j]);
                M[i * R + j] = v;
                M[j * R + i] = v;
                if (i == k + 1 && j == k + 1 && v > 0.0) rpiv = 1.0 / v;  // read after the barrier
            }
            __syncthreads();  // M and rpiv updated before the next pivot is read
        }
    }
    if (!ok) {
        // not positive definite after the ridge: report, leave the mode's
        // factor as V (Hinv = identity)
        if (threadIdx.x == 0) atomicExch(status, SPT_DEV_SINGULAR);
        for (int e = threadIdx.x; e < RR; e += blockDim.x) Hinv[e] = (e / R == e % R) ? 1.f : 0.f;
    } else {
        for (int e = threadIdx.x; e < RR; e += blockDim.x) Hinv[e] = (float)(-M[e]);
    }
    __syncthreads();  // every thread has read G before G_n is cleared
    if (zero_gram)
        for (int e = threadIdx.x; e < RR; e += blockDim.x) zero_gram[e] = 0.0;
    if (zero_colsq)
        for (int r = threadIdx.x; r < R; r += blockDim.x) zero_colsq[r] = 0.0;
}

// Threads of a hinv_kernel launch: one per pair up to 512, whole warps.
inline int hinv_threads(int R) { return std::min(512, std::max(32, (R * (R + 1) / 2 + 31) / 32 * 32)); }
inline size_t hinv_smem(int R) {
    return sizeof(double) * ((size_t)R * R + 2 * (size_t)R) + sizeof(uint32_t) * ((size_t)R * (R + 1) / 2);
}

// A32 = V Hinv, column sums of squares.  Thread (rq, cq) computes the 4 x 4
// block rows [4rq, 4rq+4) x columns [4cq, 4cq+4) of a tile of V's rows.
// Tiles of V (row stride RP + 4 floats) are double buffered with cp.async;
// Hinv sits in shared memory; each 4-wide step of k costs eight 16-byte
// shared loads for 64 FMAs.  V's columns >= R are zero (mttkrp writes them)
// and are skipped.  Sums of squares are FP32 over a thread's 4 rows of a
// tile, then FP64.
__global__ void __launch_bounds__(256) solve_kernel(const float *V, int64_t I, int ld, int R,
                                                    const float *Hinv, float *A32, double *colsq) {
    extern __shared__ __align__(16) float shs[];
    const int CT = (R + 3) / 4, RP = CT * 4;
    const int RQ = blockDim.x / CT;          // row quads per tile
    const int TROWS = 4 * RQ;
    const int SP = RP + 4;
    float *Hs = shs;                         // R x RP
    float *const vs0 = shs + R * RP;         // two tiles of TROWS x SP
    const size_t tsz = (size_t)TROWS * SP;
    __shared__ double csq[MAXR + 4];
    for (int e = threadIdx.x; e < R * RP; e += blockDim.x) {
        const int k = e / RP, c = e % RP;
        Hs[e] = c < R ? Hinv[k * R + c] : 0.f;
    }
    for (int e = threadIdx.x; e < RP; e += blockDim.x) csq[e] = 0.0;
    const int rq = threadIdx.x / CT, cq = threadIdx.x % CT;
    const bool act = rq < RQ;
    double local[4] = {0.0, 0.0, 0.0, 0.0};
    auto issue = [&](int64_t r0, float *buf) {
        for (int e = threadIdx.x; e < TROWS * CT; e += blockDim.x) {
            const int r = e / CT, q = e - r * CT;
            const bool in = r0 + r < I;
            cp_async16(buf + (size_t)r * SP + 4 * q, in ? (const void *)(V + (r0 + r) * ld + 4 * q) : V,
                       in ? 16 : 0);
        }
        cp_async_commit();
    };
    const int64_t step = (int64_t)gridDim.x * TROWS;
    int64_t r0 = (int64_t)blockIdx.x * TROWS;
    if (r0 < I) issue(r0, vs0);
    for (int k = 0; r0 < I; r0 += step, ++k) {
        const bool next = r0 + step < I;
        if (next) issue(r0 + step, vs0 + ((k + 1) & 1) * tsz);
        if (next) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncthreads();  // the tile (and Hs on the first pass) is visible
        const float *vt = vs0 + (k & 1) * tsz;
        if (act) {
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            for (int k4 = 0; k4 < CT; ++k4) {
                float vv[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 v = *reinterpret_cast<const float4 *>(&vt[(4 * rq + i) * SP + 4 * k4]);
                    vv[i][0] = v.x; vv[i][1] = v.y; vv[i][2] = v.z; vv[i][3] = v.w;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int kr = 4 * k4 + kk;
                    if (kr >= R) break;
                    const float4 h = *reinterpret_cast<const float4 *>(&Hs[kr * RP + 4 * cq]);
                    const float hh[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(vv[i][kk], hh[j], acc[i][j]);
                }
            }
            float sq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t row = r0 + 4 * rq + i;
                if (row >= I) continue;
                // columns >= R of A32 are never read
                *reinterpret_cast<float4 *>(A32 + row * ld + 4 * cq) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
#pragma unroll
                for (int j = 0; j < 4; ++j) sq[j] = fmaf(acc[i][j], acc[i][j], sq[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) local[j] += (double)sq[j];
        }
        __syncthreads();  // this buffer is refilled by the issue two tiles on
    }
    __syncthreads();  // csq zeroed (when this CTA had no tile)
    if (act)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * cq + j < R) atomicAdd(&csq[4 * cq + j], local[j]);
    __syncthreads();
    for (int e = threadIdx.x; e < R; e += blockDim.x) atomicAdd(colsq + e, csq[e]);
}

// Store the four elements of a quad in the factor's type (16 or 8 bytes).
template <typename FT> __device__ __forceinline__ void st_quad(FT *p, const float (&v)[4], float (&back)[4]);
template <> __device__ __forceinline__ void st_quad<float>(float *p, const float (&v)[4], float (&back)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
#pragma unroll
    for (int c = 0; c < 4; ++c) back[c] = v[c];
}
template <>
__device__ __forceinline__ void st_quad<__nv_bfloat16>(__nv_bfloat16 *p, const float (&v)[4], float (&back)[4]) {
    __nv_bfloat16 b[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        b[c] = __float2bfloat16_rn(v[c]);
        back[c] = __bfloat162float(b[c]);
    }
    *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(b);
}
template <> __device__ __forceinline__ void st_quad<__half>(__half *p, const float (&v)[4], float (&back)[4]) {
    __half b[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        b[c] = __float2half_rn(v[c]);
        back[c] = __half2float(b[c]);
    }
    *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(b);
}

// lambda_j = ||A32(:,j)||, store A32 * (1/lambda_j) in the factor's type
// (padding columns zero; a zero column is kept as is); on the last mode
// accumulate <X,M> = sum V(k,j) lambda_j A(k,j) (FP32 over a quad, then FP64).
// Thread t handles quad t % (ld/4) of rows t / (ld/4), +rows per pass, ...
template <typename FT>
__global__ void __launch_bounds__(256) normalize_kernel(const float *A32, const float *V, int64_t I, int ld,
                                                        int R, const double *colsq, FT *A, double *lambda,
                                                        int last, double *inner) {
    __shared__ float sinv[MAXR + 8], slam[MAXR + 8];
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const double l = sqrt(colsq[j]);
        slam[j] = (float)l;
        sinv[j] = l > 0.0 ? (float)(1.0 / l) : 1.0f;
        if (blockIdx.x == 0) lambda[j] = l;
    }
    __syncthreads();
    const int q4 = ld >> 2;
    const bool wide = q4 > (int)blockDim.x;
    const int qi = wide ? (int)threadIdx.x : (int)threadIdx.x % q4;
    const int qstep = wide ? (int)blockDim.x : q4;
    const int rr = wide ? 0 : (int)threadIdx.x / q4;
    const int rpp = wide ? 1 : (int)blockDim.x / q4;
    double local = 0.0;
    if (rr < rpp) {
        for (int64_t row = (int64_t)blockIdx.x * rpp + rr; row < I; row += (int64_t)gridDim.x * rpp) {
            for (int q = qi; q < q4; q += qstep) {
                const int64_t e = row * ld + 4 * q;
                float o[4] = {0.f, 0.f, 0.f, 0.f}, back[4];
                if (4 * q < R) {
                    const float4 a = *reinterpret_cast<const float4 *>(A32 + e);
                    const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (4 * q + c < R) o[c] = av[c] * sinv[4 * q + c];
                }
                st_quad<FT>(A + e, o, back);
                if (last && 4 * q < R) {
                    const float4 v = *reinterpret_cast<const float4 *>(V + e);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
                    float sum = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (4 * q + c < R) sum = fmaf(vv[c] * slam[4 * q + c], back[c], sum);
                    local += (double)sum;
                }
            }
        }
    }
    if (last) {
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(FULL, local, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(inner, local);
    }
}

// fit from lambda, the Grams, <X,M> and ||X||^2 (one CTA).
__global__ void fit_kernel(const double *G, int d, int R, const double *lambda, double *inner,
                           double x2, double *fit_out) {
    __shared__ double red[32];
    double local = 0.0;
    const int RR = R * R;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        double h = lambda[e / R] * lambda[e % R];
        for (int m = 0; m < d; ++m) h *= G[(int64_t)m * RR + e];
        local += h;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(FULL, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 += red[w];
        double r2 = x2 + m2 - 2.0 * (*inner);
        if (r2 < 0.0) r2 = 0.0;
        if (fit_out) *fit_out = x2 > 0.0 ? 1.0 - sqrt(r2) / sqrt(x2) : 0.0;
        *inner = 0.0;  // ready for the next iteration
    }
}

struct Ws {
    float *V, *A32, *Hinv;
    double *G, *colsq, *inner;
    double *Gp;  // partial Grams of the two-stage reduction
    int *status;
};

size_t ws_layout(spt_tensor t, int R, int ld, Ws *w, void *base) {
    int64_t imax = 1;
    for (int m = 0; m < t->d; ++m) imax = std::max(imax, t->dims[m]);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oS = take(sizeof(int));  // status word first: cp_als_status reads offset 0
    const size_t oV = take(sizeof(float) * imax * ld);
    const size_t oA = take(sizeof(float) * imax * ld);
    const size_t oH = take(sizeof(float) * R * R);
    const size_t oG = take(sizeof(double) * t->d * R * R);
    const size_t oC = take(sizeof(double) * R);
    const size_t oI = take(sizeof(double));
    const size_t oP = take(sizeof(double) * (size_t)sm_count() * gram_ctas_per_sm(R) * R * R);
    if (w && base) {
        char *b = (char *)base;
        w->V = (float *)(b + oV);
        w->A32 = (float *)(b + oA);
        w->Hinv = (float *)(b + oH);
        w->G = (double *)(b + oG);
        w->colsq = (double *)(b + oC);
        w->inner = (double *)(b + oI);
        w->Gp = (double *)(b + oP);
        w->status = (int *)(b + oS);
    }
    return off;
}

// G += A^T A.  With `partials` (room for sm_count() * gram_ctas_per_sm(R)
// R x R blocks) each CTA stores its sum there and a second kernel adds them
// in block order, so no FP64 atomics pile up on the R x R entries (the
// first form measured ~28 us of fixed cost on 608 CTAs at R = 16); without
// it each CTA adds its sum atomically.
template <typename FT>
spt_status launch_gram(const void *A, int64_t I, int ld, int R, double *G, double *partials, cudaStream_t st) {
    const GramShape g = gram_shape(R, (int)sizeof(FT));
    const int64_t tiles = (I + g.tile_rows - 1) / g.tile_rows;
    int bps = 0;
    SPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gram_kernel<FT>, g.threads, g.smem));
    bps = std::max(1, std::min(bps, gram_ctas_per_sm(R)));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count() * bps));
    gram_kernel<FT><<<blocks, g.threads, g.smem, st>>>((const FT *)A, I, ld, R, G, partials);
    SPT_LAUNCH_CHECK("gram_kernel");
    if (partials) {
        gram_reduce_kernel<<<(R * R + 7) / 8, 256, 0, st>>>(partials, blocks, R * R, G);
        SPT_LAUNCH_CHECK("gram_reduce_kernel");
    }
    return SPT_OK;
}

spt_status gram_any(spt_dtype fdt, const void *A, int64_t I, int ld, int R, double *G, double *partials,
                    cudaStream_t st) {
    if (fdt == SPT_F32) return launch_gram<float>(A, I, ld, R, G, partials, st);
    if (fdt == SPT_BF16) return launch_gram<__nv_bfloat16>(A, I, ld, R, G, partials, st);
    return launch_gram<__half>(A, I, ld, R, G, partials, st);
}

// CTAs of a solve launch over I rows in tiles of trows: as many as fit on
// the GPU at once (each keeps one tile load in flight; two CTAs per SM left
// the apply at ~40% of the copy bandwidth on 1e6 x 16 rows).
spt_status solve_grid(int64_t I, int trows, size_t smem, int *blocks) {
    int bps = 0;
    SPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, solve_kernel, 256, smem));
    *blocks = (int)std::max<int64_t>(1, std::min<int64_t>((I + trows - 1) / trows, (int64_t)sm_count() * std::max(1, bps)));
    return SPT_OK;
}

// Dynamic shared-memory limits of the CP-ALS kernels, once per device.
spt_status ensure_cpals_attrs() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    SPT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return SPT_OK;
    SPT_CUDA(cudaFuncSetAttribute(hinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hinv_smem(MAXR)));
    size_t ssm = 0;
    for (int r = 1; r <= MAXR; ++r) {
        const int ct = (r + 3) / 4, tr = 4 * (256 / ct);
        ssm = std::max(ssm, sizeof(float) * ((size_t)r * ct * 4 + (size_t)2 * tr * (ct * 4 + 4)));
    }
    SPT_CUDA(cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
    size_t gsm = 0;
    for (int r = 1; r <= MAXR; ++r) gsm = std::max(gsm, std::max(gram_shape(r, 4).smem, gram_shape(r, 2).smem));
    SPT_CUDA(cudaFuncSetAttribute(gram_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    SPT_CUDA(cudaFuncSetAttribute(gram_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    SPT_CUDA(cudaFuncSetAttribute(gram_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    done[dev] = true;
    return SPT_OK;
}

// Enqueue one iteration (no synchronisation, capturable).
spt_status enqueue_step(spt_tensor t, void *const *factors, spt_dtype fdt, int R, int ld,
                        double *lambda, double *fit_out, const Ws &w, cudaStream_t st) {
    const int d = t->d;
    {
        spt_status a = ensure_cpals_attrs();
        if (a) return a;
    }
    SPT_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * d * R * R, st));
    SPT_CUDA(cudaMemsetAsync(w.inner, 0, sizeof(double), st));
    SPT_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    // the Grams the first mode's H needs (G_0 itself is first needed after
    // mode 0's update, which recomputes it)
    for (int m = 1; m < d; ++m) {
        spt_status s = gram_any(fdt, factors[m], t->dims[m], ld, R, w.G + (size_t)m * R * R, w.Gp, st);
        if (s) return s;
    }
    for (int n = 0; n < d; ++n) {
        const int64_t In = t->dims[n];
        spt_schedule sc = default_schedule(t, n, fdt, R);
        spt_status s = launch_mttkrp(t, n, factors, fdt, R, ld, nullptr, w.V, sc, st);
        if (s) return s;
        hinv_kernel<<<1, hinv_threads(R), hinv_smem(R), st>>>(w.G, d, n, R, w.Hinv, w.G + (size_t)n * R * R, w.colsq,
                                                   w.status);
        SPT_LAUNCH_CHECK("hinv_kernel");
        const int CT = (R + 3) / 4;
        const int trows = 4 * (256 / CT);
        const size_t solve_smem = sizeof(float) * ((size_t)R * CT * 4 + (size_t)2 * trows * (CT * 4 + 4));
        int sblocks = 0;
        {
            spt_status e = solve_grid(In, trows, solve_smem, &sblocks);
            if (e) return e;
        }
        solve_kernel<<<sblocks, 256, solve_smem, st>>>(w.V, In, ld, R, w.Hinv, w.A32, w.colsq);
        SPT_LAUNCH_CHECK("solve_kernel");
        const int rpp = std::max(1, 256 / (ld / 4));  // rows per pass of a 256-thread block
        const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>((In + rpp - 1) / rpp, sm_count() * 8));
        const int last = (n == d - 1);
        if (fdt == SPT_F32)
            normalize_kernel<float><<<nblocks, 256, 0, st>>>(w.A32, w.V, In, ld, R, w.colsq,
                                                             (float *)factors[n], lambda, last, w.inner);
        else if (fdt == SPT_BF16)
            normalize_kernel<__nv_bfloat16><<<nblocks, 256, 0, st>>>(
                w.A32, w.V, In, ld, R, w.colsq, (__nv_bfloat16 *)factors[n], lambda, last, w.inner);
        else
            normalize_kernel<__half><<<nblocks, 256, 0, st>>>(w.A32, w.V, In, ld, R, w.colsq,
                                                              (__half *)factors[n], lambda, last, w.inner);
        SPT_LAUNCH_CHECK("normalize_kernel");
        s = gram_any(fdt, factors[n], In, ld, R, w.G + (size_t)n * R * R, w.Gp, st);
        if (s) return s;
    }
    fit_kernel<<<1, 256, 0, st>>>(w.G, d, R, lambda, w.inner, t->xnorm2, fit_out);
    SPT_LAUNCH_CHECK("fit_kernel");
    return SPT_OK;
}

// CUDA-graph cache: one executable graph per argument set and tensor state.
typedef std::tuple<spt_tensor, uint64_t, int, int, int, const void *, const void *, const void *,
                   const void *, const void *, const void *, const void *, const void *, const void *,
                   int>
    GraphKey;
std::mutex g_graph_mu;
std::map<GraphKey, cudaGraphExec_t> g_graphs;

}  // namespace

void drop_graphs(spt_tensor t) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (std::get<0>(it->first) == t) {
            cudaGraphExecDestroy(it->second);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace spt

using namespace spt;

extern "C" {

spt_status cp_als_workspace_size(spt_tensor t, int rank, int ld, size_t *bytes) {
    if (!t || !bytes) return fail(SPT_EINVAL, "cp_als_workspace_size: NULL argument");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_workspace_size: rank must be in [1, 128]");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "cp_als_workspace_size: bad ld");
    *bytes = ws_layout(t, rank, ld, nullptr, nullptr);
    return SPT_OK;
}

spt_status cp_als_step(spt_tensor t, void *const *factors, spt_dtype fdt, int rank, int ld,
                       double *lambda, double *fit_out, void *workspace, size_t workspace_bytes,
                       void *stream) {
    if (!t || !factors || !lambda || !workspace) return fail(SPT_EINVAL, "cp_als_step: NULL argument");
    if (!t->coalesced) return fail(SPT_ESTATE, "cp_als_step: the tensor must be created with SPT_COALESCE");
    if (t->d > SPT_MAX_KERNEL_ORDER) return fail(SPT_EUNSUPPORTED, "cp_als_step: order > 5");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_step: rank must be in [1, 128]");
    if (fdt == SPT_F64) return fail(SPT_EUNSUPPORTED, "cp_als_step: fp64 factors are supported by mttkrp only");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16) return fail(SPT_EINVAL, "cp_als_step: bad dtype");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "cp_als_step: ld must be >= rank and a multiple of 8");
    if ((uintptr_t)workspace & 255) return fail(SPT_EINVAL, "cp_als_step: workspace must be 256-byte aligned");
    for (int m = 0; m < t->d; ++m)
        if (!factors[m] || ((uintptr_t)factors[m] & 15))
            return fail(SPT_EINVAL, "cp_als_step: a factor pointer is NULL or not 16-byte aligned");
    Ws w;
    const size_t need = ws_layout(t, rank, ld, &w, workspace);
    if (workspace_bytes < need) return fail(SPT_EINVAL, "cp_als_step: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;

    const void *fp[SPT_MAX_KERNEL_ORDER] = {nullptr};
    for (int m = 0; m < t->d; ++m) fp[m] = factors[m];
    uint64_t state = 0;
    for (int m = 0; m < t->d; ++m)
        state = state * 4 + (t->blk_buf[m] ? 3 : t->sorted_buf[m] ? 2 : (t->perm[m] ? 1 : 0));
    GraphKey key(t, state, (int)fdt, rank, ld, fp[0], fp[1], fp[2], fp[3], fp[4], lambda, fit_out,
                 workspace, nullptr, t->d);
    if (st != 0) {
        cudaGraphExec_t exec = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_graph_mu);
            auto it = g_graphs.find(key);
            if (it != g_graphs.end()) exec = it->second;
        }
        if (!exec) {
            cudaGraph_t graph = nullptr;
            SPT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            spt_status s = enqueue_step(t, factors, fdt, rank, ld, lambda, fit_out, w, st);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (s) { if (graph) cudaGraphDestroy(graph); return s; }
            if (e != cudaSuccess) return cuda_fail(e, "cp_als_step: stream capture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cp_als_step: graph instantiation");
            std::lock_guard<std::mutex> lk(g_graph_mu);
            g_graphs[key] = exec;
        }
        SPT_CUDA(cudaGraphLaunch(exec, st));
        return SPT_OK;
    }
    return enqueue_step(t, factors, fdt, rank, ld, lambda, fit_out, w, st);
}

// ---- the steps of a CP-ALS mode update, one call each, for callers that
// split the rows of V (and the nonzeros) across processes or GPUs -----------

spt_status cp_als_hinv(const double *G, int order, int mode, int rank, float *hinv, int *status, void *stream) {
    if (!G || !hinv || !status) return fail(SPT_EINVAL, "cp_als_hinv: NULL argument");
    if (order < 1 || order > SPT_MAX_KERNEL_ORDER || mode < 0 || mode >= order)
        return fail(SPT_EINVAL, "cp_als_hinv: order in [1, 5] and mode in [0, order)");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_hinv: rank must be in [1, 128]");
    spt_status a = ensure_cpals_attrs();
    if (a) return a;
    cudaStream_t st = (cudaStream_t)stream;
    hinv_kernel<<<1, hinv_threads(rank), hinv_smem(rank), st>>>(G, order, mode, rank, hinv, nullptr, nullptr,
                                                                 status);
    SPT_LAUNCH_CHECK("hinv_kernel");
    return SPT_OK;
}

spt_status cp_als_apply(const float *V, int64_t rows, int ld, int rank, const float *hinv, float *A32,
                        double *colsq, void *stream) {
    if (rows < 0 || (rows > 0 && (!V || !A32)) || !hinv || !colsq) return fail(SPT_EINVAL, "cp_als_apply: NULL argument");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_apply: rank must be in [1, 128]");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "cp_als_apply: ld must be >= rank and a multiple of 8");
    if (((uintptr_t)V | (uintptr_t)A32) & 15) return fail(SPT_EINVAL, "cp_als_apply: V and A32 must be 16-byte aligned");
    spt_status a = ensure_cpals_attrs();
    if (a) return a;
    if (rows == 0) return SPT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int CT = (rank + 3) / 4;
    const int trows = 4 * (256 / CT);
    const size_t smem = sizeof(float) * ((size_t)rank * CT * 4 + (size_t)2 * trows * (CT * 4 + 4));
    int blocks = 0;
    {
        spt_status e = solve_grid(rows, trows, smem, &blocks);
        if (e) return e;
    }
    solve_kernel<<<blocks, 256, smem, st>>>(V, rows, ld, rank, hinv, A32, colsq);
    SPT_LAUNCH_CHECK("solve_kernel");
    return SPT_OK;
}

spt_status cp_als_normalize(const float *A32, const float *V, int64_t rows, int ld, int rank, const double *colsq,
                            void *A, spt_dtype fdt, double *lambda, double *inner, void *stream) {
    if (rows < 0 || (rows > 0 && (!A32 || !A)) || !colsq || !lambda)
        return fail(SPT_EINVAL, "cp_als_normalize: NULL argument");
    if ((V == nullptr) != (inner == nullptr)) return fail(SPT_EINVAL, "cp_als_normalize: V and inner go together");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_normalize: rank must be in [1, 128]");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "cp_als_normalize: ld must be >= rank and a multiple of 8");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16) return fail(SPT_EINVAL, "cp_als_normalize: bad dtype");
    if (((uintptr_t)A32 | (uintptr_t)V | (uintptr_t)A) & 15)
        return fail(SPT_EINVAL, "cp_als_normalize: A32, V and A must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int rpp = std::max(1, 256 / (ld / 4));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + rpp - 1) / rpp, sm_count() * 8));
    const int last = inner ? 1 : 0;
    if (fdt == SPT_F32)
        normalize_kernel<float><<<blocks, 256, 0, st>>>(A32, V, rows, ld, rank, colsq, (float *)A, lambda, last, inner);
    else if (fdt == SPT_BF16)
        normalize_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(A32, V, rows, ld, rank, colsq, (__nv_bfloat16 *)A,
                                                                lambda, last, inner);
    else
        normalize_kernel<__half><<<blocks, 256, 0, st>>>(A32, V, rows, ld, rank, colsq, (__half *)A, lambda, last,
                                                         inner);
    SPT_LAUNCH_CHECK("normalize_kernel");
    return SPT_OK;
}

spt_status cp_als_gram(const void *A, int64_t rows, int ld, int rank, spt_dtype fdt, double *G, void *stream) {
    if (rows < 0 || (rows > 0 && !A) || !G) return fail(SPT_EINVAL, "cp_als_gram: NULL argument");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_gram: rank must be in [1, 128]");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "cp_als_gram: ld must be >= rank and a multiple of 8");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16) return fail(SPT_EINVAL, "cp_als_gram: bad dtype");
    if ((uintptr_t)A & 15) return fail(SPT_EINVAL, "cp_als_gram: A must be 16-byte aligned");
    spt_status a = ensure_cpals_attrs();
    if (a) return a;
    if (rows == 0) return SPT_OK;
    return gram_any(fdt, A, rows, ld, rank, G, nullptr, (cudaStream_t)stream);
}

spt_status cp_als_fit(const double *G, int order, int rank, const double *lambda, double *inner, double xnorm2,
                      double *fit, void *stream) {
    if (!G || !lambda || !inner || !fit) return fail(SPT_EINVAL, "cp_als_fit: NULL argument");
    if (order < 1 || order > SPT_MAX_KERNEL_ORDER) return fail(SPT_EINVAL, "cp_als_fit: order in [1, 5]");
    if (rank < 1 || rank > MAXR) return fail(SPT_EUNSUPPORTED, "cp_als_fit: rank must be in [1, 128]");
    fit_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(G, order, rank, lambda, inner, xnorm2, fit);
    SPT_LAUNCH_CHECK("fit_kernel");
    return SPT_OK;
}

spt_status cp_als_status(void *workspace, void *stream) {
    if (!workspace) return fail(SPT_EINVAL, "cp_als_status: NULL workspace");
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    SPT_CUDA(cudaMemcpyAsync(&h, workspace, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPT_CUDA(cudaStreamSynchronize(st));
    if (h == SPT_DEV_SINGULAR)
        return fail(SPT_ESINGULAR, "cp_als_step: a Gram-Hadamard matrix was not positive definite");
    if (h) return fail(SPT_ECUDA, "cp_als_step: device status " + std::to_string(h));
    return SPT_OK;
}

}  // extern "C"

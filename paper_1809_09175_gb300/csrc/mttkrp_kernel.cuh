// mttkrp_kernel.cuh -- the sparse COO MTTKRP kernel (Sec. 3 eq. mttkrp).
//
//   out(k, j) = lambda_j * sum_{i : l_in = k} x_i * prod_{m != n} A^(m)(l_im, j)
//
// Work decomposition (GB300 mapping of the paper's league/team/vector levels,
// Sec. 4 Tab. "Levels of Parallelism"):
//  * Each warp of a persistent grid owns a contiguous range of chunks of
//    `npw` consecutive nonzeros of the traversal order.  A chunk's
//    nonzeros are staged into the warp's shared memory with 1-D bulk copies
//    (cp.async.bulk, mbarrier completion), double buffered, so the next chunk
//    streams in while this one is computed.
//  * The warp is split into G = 32/L groups of L lanes.  Group g walks the
//    nonzeros [g*S, g*S+S) of the chunk in order (the paper's NZPTM block,
//    Fig. MTTKRP-C); lane l of the group owns 4-column chunks of the rank
//    block (the paper's vector lanes over j, Fig. MTTKRP-B), loading the d-1
//    factor rows with coalesced vector loads (16 bytes per chunk for fp32,
//    8 for 16-bit factors) and keeping the running row sum in registers (the
//    paper's TinyVec).
//  * Scatter:
//      M_ATOMIC  storage order (coordinate arrays staged one by one); a
//                group's running sum is added atomically (16-byte vector red)
//                whenever its row changes (Fig. MTTKRP-B with merging of
//                equal consecutive rows).  The mode's hottest rows (a list
//                made when the tensor is created) are the exception: their
//                flushes are added into a per-CTA copy of those rows in
//                shared memory (found through a small hash table), which the
//                CTA adds to the output once at the end.  A row holding a
//                large share of the nonzeros then takes one chain of adds per
//                CTA instead of one serialised global chain as long as its
//                nonzero count: faster, and without the rounding drift of
//                millions of fp32 adds into one running value.
//      M_SORTED  mode-n order from the mode-sorted copy, whose nonzeros are
//                packed records {row, other coordinates, value} (one bulk copy
//                and one vector shared load per nonzero);
//      M_PERM    storage order walked through the permutation (Fig. MTTKRP-C):
//                the permutation is staged, coordinates and values gathered.
//                For both, a group writes a finished row with a plain store;
//                the first and last run of every group are combined across
//                the warp with shuffles (a log-step segmented scan over the
//                groups' tail runs, after which each group writes the runs
//                that end in it), and the last open run is carried in shared memory
//                into the warp's next chunk, so only the first and last row
//                of the warp's whole range are added atomically: only those
//                rows can be shared with other warps.
//      M_PRIVATE storage order like M_ATOMIC, but every row flush is an
//                atomic add into a private copy of the output held in shared
//                memory (the privatised scatter the paper proposes for short
//                modes, Sec. 8).  When one CTA's shared memory cannot hold
//                I_n rows, a thread-block cluster of K CTAs splits them
//                (row k lives in CTA k mod K, local row k / K) and adds reach
//                the owner through distributed shared memory.  After the
//                cluster barrier each CTA adds its rows to the output with
//                16-byte vector atomics.
//  * Columns: rank block rb covers columns [rb*L*C*VEC, ...); lane l's chunk
//    c starts at column rb*L*C*VEC + (c*L + l)*VEC.  Columns >= R are
//    computed from the factors' padding and written as zeros.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace spt {

enum MttkrpMode { M_ATOMIC = 0, M_SORTED = 1, M_PERM = 2, M_PRIVATE = 3 };

// Words of one packed record of the mode-sorted copy: {row, d-1 other
// coordinates, value} = d+1 words, padded to 2, 4 or 6 for vector loads.
__host__ __device__ constexpr int record_words(int d) {
    return d + 1 <= 2 ? 2 : (d + 1 <= 4 ? 4 : (d + 1 <= 6 ? 6 : ((d + 2) & ~1)));
}

struct MttkrpParams {
    const int32_t *rows;     // M_ATOMIC / M_PERM: mode-n coordinates, storage order
    const int32_t *oidx[4];  // M_ATOMIC / M_PERM: coordinates of the other modes
    const float *vals;       // M_ATOMIC / M_PERM: values
    const int32_t *perm;     // M_PERM: traversal position -> storage position
    const int32_t *rec;      // M_SORTED: packed records in mode-n order; M_PERM, nullable: the
                             // storage-order records (all d coordinates, then the value)
    const void *fac[4];      // factor matrices of the other modes
    int fld;                 // factor row stride (elements)
    const void *lambda;      // nullable; accumulator type (float, double for fp64)
    void *out;               // I_n x old accumulator type (float, double for fp64), zeroed first
    int64_t old;
    int64_t nnz;
    int R;
    int rb_cols;  // columns per rank block = L*C*VEC
    int n_rb;     // number of rank blocks
    int log2L;    // lanes per nonzero = 1 << log2L
    int S;        // nonzeros per group per chunk
    int npw;      // nonzeros per warp chunk = (32 >> log2L) * S, a multiple of 4
    int64_t nchunks;
    int *err;     // device status word
    uint32_t wait_tries;  // try budget of a staging wait (the drain after a
                          // timeout always uses the full SPT_WAIT_TRIES)
    // M_ATOMIC: the hot rows held in shared memory (nhot = 0: none)
    const int32_t *hot_rows;  // nhot row ids, hottest first
    int nhot;
    int hot_log2T;            // hash table of 1 << hot_log2T slots (>= 2 nhot)
    int accum;                // M_SORTED: every row sum is added to the output (vector atomic
                              // adds), none stored: one launch of several over the groups of
                              // an L2-blocked copy
    int nrep;                 // M_ATOMIC: copies of the output (a power of two, >= 1); CTA b
    int64_t rep_stride;       // adds into copy b & (nrep - 1), rep_stride elements apart
                              // (out is then a scratch summed into the output afterwards)
    // M_PRIVATE: the private output copy in shared memory
    int In;       // rows of the output (mode length)
    int pld;      // row stride of the shared-memory copy (private or hot rows) in
                  // accumulator elements, R rounded up to 4
    int log2K;    // cluster size K = 1 << log2K CTAs share the rows
    int prows;    // private rows per CTA = ceil(In / K)
    // deterministic sums (sorted traversal with the run carry): the first and
    // last row of warp gw's range go to slots 2 gw and 2 gw + 1 (row ids,
    // partial rows of stride old) instead of atomics; a fix-up kernel adds the
    // slots of each row in an order fixed by the slot layout (DET kernels only)
    int *det_rows;
    void *det_vals;
    // generalised CP gradient (gcp kernels only)
    const void *fac_n;   // the mode's own factor A^(n): the model value needs it
    int loss;            // 0 Poisson (stored part), 1 Bernoulli-logit, 2 Gaussian
    double *loss_out;    // nullable: sum of the stored entries' loss terms
    int mode;            // n (M_PERM over storage-order records: the output row's word)
};

__device__ __forceinline__ uint4 ldg16(const void *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

__device__ __forceinline__ void red_add4(float *dst, const float *v) {
    atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void red_add4(double *dst, const double *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(dst + q, v[q]);
}
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return fmaf(a, b, c); }

// Two fp32 multiplies / FMAs in one packed instruction (mul / fma .rn.f32x2,
// sm_100 and later); each half rounds exactly as the scalar operation, so
// results are bit-identical to the scalar form.  Measured on the sorted
// traversal: 3-way fp32 R=16 +2.7%, 4-way bf16 R=64 +2.3%, 4-way fp32 R=64
// -2.2% (there the scalar form stays).  0 turns it off everywhere.
#ifndef SPT_PACKED_FMA
#define SPT_PACKED_FMA 1
#endif
__device__ __forceinline__ void mul2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1, float c0,
                                     float c1) {
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%6, %7};\n\tfma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}
__device__ __forceinline__ double fma_acc(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ void store4(float *dst, const float *v) {
    *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double *dst, const double *v) {
    reinterpret_cast<double2 *>(dst)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(dst)[1] = make_double2(v[2], v[3]);
}

// 0: every chunk takes the group-contiguous walk (build variant for comparisons)
#ifndef SPT_SINGLE_ROW_CHUNKS
#define SPT_SINGLE_ROW_CHUNKS 1
#endif

// Register cap: small column blocks fit two 512-thread CTAs (<= 64 registers).
#ifndef SPT_MTTKRP_MINBLOCKS
#define SPT_MTTKRP_MINBLOCKS 2
#endif
template <typename FT, int C> struct MinBlocks {
    static constexpr int value = (Elem<FT>::VEC * C <= 4 && Elem<FT>::BYTES <= 4) ? SPT_MTTKRP_MINBLOCKS : 1;
};

// Open row sum carried from one chunk to the next by a warp that walks a
// contiguous range of chunks (one rank block), kept in the warp's shared
// memory between chunks: a 16-byte header (the carried row, then the first
// and last row of the warp's range) and C x 4 accumulators of AB bytes for
// each of the L column slices (every group holds the same slices).
__host__ __device__ constexpr int carry_bytes(int C, int L, int AB) { return 16 + 4 * AB * C * L; }

// First and last mode-n coordinate of the staged chunk.
template <int D1, int MODE>
__device__ __forceinline__ void chunk_bounds(const MttkrpParams &p, const int32_t *buf, int n, int &b0,
                                             int &b1) {
    constexpr int REC = record_words(D1 + 1);
    if (MODE == M_SORTED) {
        b0 = buf[0];
        b1 = buf[(n - 1) * REC];
    } else if (MODE == M_PERM) {
        b0 = __ldg(p.rows + buf[0]);
        b1 = __ldg(p.rows + buf[n - 1]);
    } else {
        b0 = b1 = -1;
    }
}

// Shared-memory layout of the atomic scatter's hot rows: nhot rows of pld
// accumulators, then the hash table's keys (row ids, -1 = empty) and values
// (slot of the row), 1 << hot_log2T of each.
__host__ __device__ inline size_t hot_smem_bytes(int nhot, int pld, int ab, int log2T) {
    return nhot > 0 ? (size_t)nhot * pld * ab + (size_t)2 * 4 * (1u << log2T) : 0;
}

// Slot of `row` among the hot rows, or -1 (linear probing; the table is at
// most half full, so a miss stops at an empty slot within a few probes).
__device__ __forceinline__ int hot_slot(const int *hkey, int log2T, int row) {
    const unsigned mask = (1u << log2T) - 1u;
    unsigned h = ((unsigned)row * 0x9E3779B1u) >> (32 - log2T);
    for (unsigned q = 0; q <= mask; ++q) {
        const int k = hkey[h];
        if (k == row) return hkey[(1u << log2T) + h];
        if (k < 0) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Compute one staged chunk of n nonzeros (n <= npw) for every rank block:
// gather, multiply, segmented accumulate and write (see the file comment).
// Rows b0 and b1 may be shared with other warps and are added atomically;
// every other finished row is stored.  With `carry` (single rank block), the
// chunk's last open run is handed over instead of written, the carried run of
// the previous chunk joins this chunk's first run, and the shared rows are the
// range's first and last rows from the carry header.
template <typename FT, int C, int D1, int MODE, bool GCP = false, bool CLAMP = false, bool DET = false>
__device__ __forceinline__ void mttkrp_chunk(const MttkrpParams &p, const int32_t *buf, int n, int b0,
                                             int b1, unsigned char *carry, typename Elem<FT>::Acc *priv,
                                             double *lacc = nullptr) {
    using E = Elem<FT>;
    using Raw = typename E::Raw;
    using AT = typename E::Acc;
    constexpr int VEC = E::VEC;
    constexpr int DA = D1 > 0 ? D1 : 1;
    // gathered rows per nonzero: the d-1 other factors, plus the own factor's
    // row for the generalised CP model value (slot D1)
    constexpr int NR = GCP ? D1 + 1 : DA;
    constexpr int REC = record_words(D1 + 1);
    constexpr int LOADS = NR * C;
    constexpr int U = (LOADS <= 2) ? 2 : 1;
    constexpr unsigned FULL = 0xffffffffu;
    // packed fp32 products (fp32 accumulators; 16-bit factors, or fp32 ones of
    // orders <= 3); bit-identical to the scalar form
    constexpr bool PACKED = SPT_PACKED_FMA && std::is_same<AT, float>::value && VEC % 2 == 0 &&
                            (E::BYTES == 2 || D1 <= 2);
    const int lane = threadIdx.x & 31;
    const int npw = p.npw;
    const int log2L = p.log2L;
    const int L = 1 << log2L;
    const int G = 32 >> log2L;
    const int g = lane >> log2L;
    const int l = lane & (L - 1);
    const int S = p.S;
    const int rstride = p.fld * (int)sizeof(FT);  // bytes per factor row (< 2^31, checked on the host)

    const int e0 = g * S;
    const int cnt = max(0, min(S, n - e0));

    for (int rb = 0; rb < p.n_rb; ++rb) {
        int col[C], nv[C];
        AT lam[C][VEC];
        const char *fb[NR][C];  // this lane's column chunk of each factor
#pragma unroll
        for (int c = 0; c < C; ++c) {
            col[c] = rb * p.rb_cols + (c * L + l) * VEC;
            nv[c] = max(0, min(VEC, p.R - col[c]));
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                lam[c][v] = (p.lambda && v < nv[c]) ? __ldg(reinterpret_cast<const AT *>(p.lambda) + col[c] + v)
                                                     : (AT)1;
            // CLAMP: a chunk wholly past column R gathers column 0 instead (in
            // bounds, loaded unpredicated, its sums never written), so lanes
            // past R do not make the gathers diverge
            const int64_t cb0 = (int64_t)(CLAMP && nv[c] == 0 ? 0 : col[c]) * sizeof(FT);
#pragma unroll
            for (int m = 0; m < D1; ++m) fb[m][c] = reinterpret_cast<const char *>(p.fac[m]) + cb0;
            if (GCP) fb[NR - 1][c] = reinterpret_cast<const char *>(p.fac_n) + cb0;
        }

        AT acc[C][VEC], facc[C][VEC];
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = facc[c][v] = (AT)0;
        int cur = -1, frow = -1;
        bool fclosed = false;

        // emit a finished row sum: atomic for shared rows, plain store otherwise;
        // dslot: the range's boundary slot of a shared row (0 first, 1 last)
        auto write_row = [&](int row, AT (&a)[C][VEC], bool atomic, int dslot = -1) {
            if (MODE == M_PRIVATE) {  // add into the owning CTA's private copy
                const int K = 1 << p.log2K;
                AT *prow = priv + (int64_t)(row >> p.log2K) * p.pld;
                const uint32_t owner = (uint32_t)(row & (K - 1));
#pragma unroll
                for (int c = 0; c < C; ++c) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        if (v >= nv[c]) continue;
                        const AT w = a[c][v] * lam[c][v];
                        const uint32_t a = smem_u32(prow + col[c] + v);
                        if (K == 1)
                            red_add_shared(a, w);
                        else
                            red_add_cluster(mapa_shared(a, owner), w);
                    }
                }
                return;
            }
            if (MODE == M_ATOMIC && priv) {  // a hot row: add into this CTA's shared copy
                const int slot = hot_slot(reinterpret_cast<const int *>(priv + (int64_t)p.nhot * p.pld),
                                          p.hot_log2T, row);
                if (slot >= 0) {
                    AT *hrow = priv + (int64_t)slot * p.pld;
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            if (v < nv[c]) red_add_shared(smem_u32(hrow + col[c] + v), a[c][v] * lam[c][v]);
                    return;
                }
            }
            AT *dst = reinterpret_cast<AT *>(p.out) + (int64_t)row * p.old;
            if (MODE == M_ATOMIC) dst += (int64_t)(blockIdx.x & (p.nrep - 1)) * p.rep_stride;
            if (MODE == M_SORTED && p.accum) atomic = true;  // rows add up across launches
            if (DET && atomic && dslot >= 0) {  // deterministic: this warp's slot
                const int slot = 2 * (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) + dslot;
                dst = reinterpret_cast<AT *>(p.det_vals) + (int64_t)slot * p.old;
                if (l == 0) p.det_rows[slot] = row;
                atomic = false;
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (nv[c] == 0) continue;
                AT w[VEC];  // columns >= R hold padding products: write zeros
#pragma unroll
                for (int v = 0; v < VEC; ++v) w[v] = v < nv[c] ? a[c][v] * lam[c][v] : (AT)0;
#pragma unroll
                for (int q = 0; q < VEC; q += 4) {
                    if (atomic) red_add4(dst + col[c] + q, w + q);
                    else store4(dst + col[c] + q, w + q);
                }
            }
        };

        // load one nonzero's row, value and its d-1 factor-row chunks
        // own_row = false: the generalised CP's own-factor row is not loaded
        // (a single-row chunk loads it once for all its nonzeros)
        auto fetch = [&](int e, int &row, float &x, Raw (&rw)[NR][C], bool own_row = true) {
            int r[DA];
            if (MODE == M_SORTED) {
                int w[REC];
                const int32_t *rp = buf + e * REC;
                if (REC == 4) {
                    const int4 q = *reinterpret_cast<const int4 *>(rp);
                    w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
                } else {
#pragma unroll
                    for (int h = 0; h < REC; h += 2) {
                        const int2 q = *reinterpret_cast<const int2 *>(rp + h);
                        w[h] = q.x;
                        w[h + 1] = q.y;
                    }
                }
                row = w[0];
#pragma unroll
                for (int m = 0; m < D1; ++m) r[m] = w[1 + m];
                x = __int_as_float(w[D1 + 1]);
            } else if (MODE == M_PERM) {
                const int q = buf[e];
                if (p.rec) {  // one storage-order record per nonzero: its coordinates, then the value
                    int w[REC];
                    const int32_t *rp = p.rec + (int64_t)q * REC;
                    if (REC == 4) {
                        const int4 v = __ldg(reinterpret_cast<const int4 *>(rp));
                        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
                    } else {
#pragma unroll
                        for (int h = 0; h < REC; h += 2) {
                            const int2 v = __ldg(reinterpret_cast<const int2 *>(rp + h));
                            w[h] = v.x;
                            w[h + 1] = v.y;
                        }
                    }
                    // word n is the row; the others in increasing mode order
                    row = w[0];
#pragma unroll
                    for (int m = 1; m <= D1; ++m)
                        if (m == p.mode) row = w[m];
#pragma unroll
                    for (int m = 0; m < D1; ++m) r[m] = m < p.mode ? w[m] : w[m + 1];
                    x = __int_as_float(w[D1 + 1]);
                } else {
                    row = __ldg(p.rows + q);
                    x = __ldg(p.vals + q);
#pragma unroll
                    for (int m = 0; m < D1; ++m) r[m] = __ldg(p.oidx[m] + q);
                }
            } else {
                row = buf[e];
                x = __int_as_float(buf[(D1 + 1) * npw + e]);
#pragma unroll
                for (int m = 0; m < D1; ++m) r[m] = buf[(1 + m) * npw + e];
            }
#pragma unroll
            for (int m = 0; m < D1; ++m) {
#pragma unroll
                for (int c = 0; c < C; ++c)
                    rw[m][c] = (CLAMP || nv[c] > 0) ? E::load(fb[m][c] + (int64_t)r[m] * rstride) : Raw{};
            }
            if (GCP && own_row) {
#pragma unroll
                for (int c = 0; c < C; ++c)
                    rw[NR - 1][c] = (CLAMP || nv[c] > 0) ? E::load(fb[NR - 1][c] + (int64_t)row * rstride) : Raw{};
            }
        };
        float lsum = 0.0f;  // generalised CP: this lane's loss terms of the chunk (fp32)
        // multiply out one nonzero and fold it into the running row sum;
        // `vote`: every lane of the warp runs this step (uniform fast path)
        auto step = [&](int row, float x, const Raw (&rw)[NR][C], bool vote) {
            AT part[C][VEC], fl[C][VEC];  // x * first D1-1 factors; last factor
            if constexpr (GCP) {
                // t = prod of the other factors' rows; m = <A^(n)(row,:), t>
                // summed over the group's lanes; the row sum gathers
                // df/dm(x, m) * t (part = df/dm, fl = t)
                AT dot = (AT)0;
#pragma unroll
                for (int c = 0; c < C; ++c) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) fl[c][v] = (AT)1;
#pragma unroll
                    for (int m = 0; m < D1; ++m) {
                        AT f[VEC];
                        E::widen(rw[m][c], f);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) fl[c][v] *= f[v];
                    }
                    AT an[VEC];
                    E::widen(rw[NR - 1][c], an);
#pragma unroll
                    for (int v = 0; v < VEC; ++v)
                        if (v < nv[c]) dot = fma_acc(fl[c][v], an[v], dot);
                }
                const unsigned gmask = L == 32 ? FULL : (((1u << L) - 1u) << (g * L));
                for (int o = 1; o < L; o <<= 1) dot += __shfl_xor_sync(gmask, dot, o);
                const float mv = (float)dot;
                float y, fv;
                // fast-math intrinsics: a few ulp, far inside the 2e-5 gradient bound
                if (p.loss == 0) {  // Poisson: the stored entry's part of 1 - x/m
                    y = -__fdividef(x, mv);
                    fv = -x * __logf(mv);
                } else if (p.loss == 1) {  // Bernoulli, logit link
                    const float e = __expf(-fabsf(mv));  // log(1 + e^m) = max(m, 0) + log(1 + e^-|m|)
                    y = (mv >= 0.0f ? __fdividef(1.0f, 1.0f + e) : __fdividef(e, 1.0f + e)) - x;
                    fv = fmaxf(mv, 0.0f) + __logf(1.0f + e) - x * mv;
                } else {  // Gaussian
                    y = 2.0f * (mv - x);
                    fv = (mv - x) * (mv - x);
                }
                if (l == 0) lsum += fv;
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) part[c][v] = (AT)y;
            } else {
#pragma unroll
            for (int c = 0; c < C; ++c) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) part[c][v] = (AT)x;
#pragma unroll
                for (int m = 0; m + 1 < D1; ++m) {
                    AT f[VEC];
                    E::widen(rw[m][c], f);
                    if constexpr (PACKED) {
#pragma unroll
                        for (int v = 0; v < VEC; v += 2)
                            mul2(part[c][v], part[c][v + 1], part[c][v], part[c][v + 1], f[v], f[v + 1]);
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) part[c][v] *= f[v];
                    }
                }
                if (D1 > 0) E::widen(rw[DA - 1][c], fl[c]);
            }
            }
            const bool ch = row != cur;
            const bool any = vote ? __any_sync(FULL, ch) : ch;
            if (any && ch) {
                if (cur >= 0) {
                    if (MODE == M_ATOMIC || MODE == M_PRIVATE) {
                        write_row(cur, acc, true);
                    } else if (!fclosed) {
                        fclosed = true;
                        frow = cur;
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) facc[c][v] = acc[c][v];
                    } else {
                        write_row(cur, acc, false);  // row lies inside this group's block
                    }
                }
                cur = row;
                if constexpr (PACKED && D1 > 0) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; v += 2)
                            mul2(acc[c][v], acc[c][v + 1], part[c][v], part[c][v + 1], fl[c][v], fl[c][v + 1]);
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            acc[c][v] = D1 > 0 ? part[c][v] * fl[c][v] : part[c][v];
                }
            } else {
                if constexpr (PACKED && D1 > 0) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; v += 2)
                            fma2(acc[c][v], acc[c][v + 1], part[c][v], part[c][v + 1], fl[c][v], fl[c][v + 1],
                                 acc[c][v], acc[c][v + 1]);
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            acc[c][v] = D1 > 0 ? fma_acc(part[c][v], fl[c][v], acc[c][v])
                                               : acc[c][v] + part[c][v];
                }
            }
        };

        const bool single_row = SPT_SINGLE_ROW_CHUNKS && MODE == M_SORTED && !DET && carry && n == npw &&
                                buf[0] == buf[(n - 1) * REC];
#if SPT_SINGLE_ROW_CHUNKS
        if (single_row) {
            // A full chunk inside one row (a long slice): the groups take
            // consecutive nonzeros (t*G + g), so factor rows that neighbours
            // repeat -- the mode-sorted copy orders a slice by the other
            // modes -- share one load in a warp instruction; then the
            // groups' sums are added by a shuffle butterfly and join the run
            // carried from the previous chunk.  The generalised CP's own row
            // is the same for every nonzero: loaded once.
            Raw own[C];
            if (GCP) {
#pragma unroll
                for (int c = 0; c < C; ++c)
                    own[c] = (CLAMP || nv[c] > 0) ? E::load(fb[NR - 1][c] + (int64_t)buf[0] * rstride) : Raw{};
            }
            for (int t = 0; t + U <= S; t += U) {
                int rowu[U];
                float xu[U];
                Raw raw[U][NR][C];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    fetch((t + u) * G + g, rowu[u], xu[u], raw[u], false);
                    if (GCP) {
#pragma unroll
                        for (int c = 0; c < C; ++c) raw[u][NR - 1][c] = own[c];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) step(rowu[u], xu[u], raw[u], true);
            }
            for (int t = S - S % U; t < S; ++t) {
                int row;
                float x;
                Raw rw[NR][C];
                fetch(t * G + g, row, x, rw, false);
                if (GCP) {
#pragma unroll
                    for (int c = 0; c < C; ++c) rw[NR - 1][c] = own[c];
                }
                step(row, x, rw, true);
            }
            if (GCP) *lacc += (double)lsum;  // the loss terms of the chunk's nonzeros
            for (int off = L; off < 32; off <<= 1)
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][v] += __shfl_xor_sync(FULL, acc[c][v], off);
            int *crow_p = reinterpret_cast<int *>(carry);
            AT *cacc_p = reinterpret_cast<AT *>(carry + 16) + l * (C * VEC);
            const int crow = *crow_p;
            AT cin[C][VEC];
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) cin[c][v] = cacc_p[c * VEC + v];
            if (crow == cur) {
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][v] += cin[c][v];
            } else if (crow >= 0 && g == 0) {  // the carried run ended before this chunk
                write_row(crow, cin, crow == crow_p[1] || crow == crow_p[2], crow == crow_p[2]);
            }
            __syncwarp();  // every lane has read the carry
            if (g == 0) {
                if (l == 0) *crow_p = cur;
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) cacc_p[c * VEC + v] = acc[c][v];
            }
            continue;  // the only rank block
        }
#endif
        if (n == npw) {
            // full chunk: every group walks exactly S nonzeros, U at a time
            int t = 0;
            for (; t + U <= S; t += U) {
                int rowu[U];
                float xu[U];
                Raw raw[U][NR][C];
#pragma unroll
                for (int u = 0; u < U; ++u) fetch(e0 + t + u, rowu[u], xu[u], raw[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) step(rowu[u], xu[u], raw[u], true);
            }
            for (; t < S; ++t) {
                int row;
                float x;
                Raw rw[NR][C];
                fetch(e0 + t, row, x, rw);
                step(row, x, rw, true);
            }
        } else {
            // the tensor's last, ragged chunk: groups hold different counts
            for (int t = 0; t < cnt; ++t) {
                int row;
                float x;
                Raw rw[NR][C];
                fetch(e0 + t, row, x, rw);
                step(row, x, rw, false);
            }
        }

        if (GCP) *lacc += (double)lsum;
        if (MODE == M_ATOMIC || MODE == M_PRIVATE) {
            if (cur >= 0) write_row(cur, acc, true);
        } else {
            // Segmented combine of the groups' open runs.  Every group holds
            // a tail run (cur, acc) and, if it saw a row change, a closed
            // head run (frow, facc); rows between them are already written.
            int *crow_p = reinterpret_cast<int *>(carry);
            AT *cacc_p = carry ? reinterpret_cast<AT *>(carry + 16) + l * (C * VEC) : nullptr;
            const int s0 = carry ? crow_p[1] : b0, s1 = carry ? crow_p[2] : b1;
            auto shared_row = [&](int row) { return row == s0 || row == s1; };
            if (n == npw && G > 1) {
                // Full chunk (every group non-empty): a log-step segmented
                // scan of the tails over the groups, then each group writes
                // the runs that end in it.  A group's tail continues the
                // previous group's chain unless it has a head or a new row.
                const int crow = carry ? *crow_p : -1;
                const int first = fclosed ? frow : cur;
                int prevrow = __shfl_up_sync(FULL, cur, L);
                if (g == 0) prevrow = crow;
                AT cin[C][VEC], T[C][VEC];
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        cin[c][v] = carry ? cacc_p[c * VEC + v] : (AT)0;
                        T[c][v] = acc[c][v];
                    }
                int f = (fclosed || cur != prevrow) ? 1 : 0;
                if (g == 0 && !f) {  // the carried run continues into group 0's tail
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) T[c][v] += cin[c][v];
                }
                if (g == 0 && crow >= 0 && first != crow) write_row(crow, cin, shared_row(crow), crow == s1);
                for (int off = 1; off < G; off <<= 1) {
                    const int fu = __shfl_up_sync(FULL, f, off * L);
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const AT tu = __shfl_up_sync(FULL, T[c][v], off * L);
                            if (g >= off && !f) T[c][v] += tu;
                        }
                    if (g >= off) f |= fu;
                }
                // the chain ending in group g-1 (the carry for group 0)
                AT Sp[C][VEC];
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        const AT su = __shfl_up_sync(FULL, T[c][v], L);
                        Sp[c][v] = g == 0 ? cin[c][v] : su;
                    }
                const int nf = __shfl_down_sync(FULL, first, L);  // first row of group g+1
                if (fclosed) {  // the head joins the chain ending before it if the rows agree
                    if (frow == prevrow) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) facc[c][v] += Sp[c][v];
                    }
                    write_row(frow, facc, shared_row(frow), frow == s1);
                }
                if (g < G - 1) {
                    if (nf != cur) write_row(cur, T, shared_row(cur), cur == s1);  // the chain ends here
                } else if (!carry) {
                    write_row(cur, T, shared_row(cur), cur == s1);
                }
                if (carry) {
                    __syncwarp();  // every lane has read the carry
                    if (g == G - 1) {
                        if (l == 0) *crow_p = cur;
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) cacc_p[c * VEC + v] = T[c][v];
                    }
                }
                continue;  // next rank block
            }
            // Ragged chunk or one group: the groups' runs in group order.
            // Every lane tracks the running (orow, oacc) for its columns;
            // group 0's lanes perform the writes.
            AT oacc[C][VEC];
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) oacc[c][v] = carry ? cacc_p[c * VEC + v] : (AT)0;
            int orow = carry ? *crow_p : -1;
            const bool writer = (g == 0);
            auto emit = [&](int row, AT (&a)[C][VEC]) {
                if (writer) write_row(row, a, shared_row(row), row == s1);
            };
            for (int g2 = 0; g2 < G; ++g2) {
                const int srcl = (g2 << log2L) | l;
                const int scur = __shfl_sync(FULL, cur, srcl);
                if (scur < 0) break;  // this and later groups got no nonzeros
                const int sfc = __shfl_sync(FULL, (int)fclosed, srcl);
                const int sfrow = __shfl_sync(FULL, frow, srcl);
                AT F[C][VEC], A[C][VEC];
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        F[c][v] = __shfl_sync(FULL, facc[c][v], srcl);
                        A[c][v] = __shfl_sync(FULL, acc[c][v], srcl);
                    }
                if (sfc) {
                    if (orow == sfrow) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) F[c][v] += oacc[c][v];
                    } else if (orow >= 0) {
                        emit(orow, oacc);
                    }
                    emit(sfrow, F);
                    orow = scur;
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) oacc[c][v] = A[c][v];
                } else if (orow == scur) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) oacc[c][v] += A[c][v];
                } else {
                    if (orow >= 0) emit(orow, oacc);
                    orow = scur;
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) oacc[c][v] = A[c][v];
                }
            }
            if (carry) {
                __syncwarp();  // every lane has read the carry
                if (lane == 0) *crow_p = orow;
                if (g == 0) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) cacc_p[c * VEC + v] = oacc[c][v];
                }
            } else if (orow >= 0) {
                emit(orow, oacc);
            }
        }
    }
}

// Atomically add a carried row sum (rank block 0) to the output.
template <typename FT, int C, bool DET = false>
__device__ __forceinline__ void flush_carry(const MttkrpParams &p, const unsigned char *carry) {
    constexpr int VEC = Elem<FT>::VEC;
    using AT = typename Elem<FT>::Acc;
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.log2L;
    const int row = *reinterpret_cast<const int *>(carry);
    if ((lane >> p.log2L) != 0 || row < 0) return;  // group 0 writes
    const int l = lane & (L - 1);
    const AT *acc = reinterpret_cast<const AT *>(carry + 16) + l * (C * VEC);
    AT *dst = reinterpret_cast<AT *>(p.out) + (int64_t)row * p.old;
    constexpr bool det = DET;  // the range's last row goes to the warp's slot 1
    if (det) {
        const int slot = 2 * (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) + 1;
        dst = reinterpret_cast<AT *>(p.det_vals) + (int64_t)slot * p.old;
        if (l == 0) p.det_rows[slot] = row;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = (c * L + l) * VEC;
        const int nv = max(0, min(VEC, p.R - col));
        if (nv == 0) continue;
        AT w[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v)
            w[v] = v < nv ? acc[c * VEC + v] * (p.lambda ? __ldg(reinterpret_cast<const AT *>(p.lambda) + col + v)
                                                          : (AT)1)
                          : (AT)0;
#pragma unroll
        for (int q = 0; q < VEC; q += 4) {
            if (det) store4(dst + col + q, w + q);
            else red_add4(dst + col + q, w + q);
        }
    }
}

// Staged 32-bit words per nonzero of a traversal mode.
template <int D1, int MODE> struct Staging {
    static constexpr int NARR = (MODE == M_PERM) ? 1 : (D1 + 2);  // SoA arrays staged
    static constexpr int WPE = (MODE == M_SORTED) ? record_words(D1 + 1) : NARR;
};

// Bytes of the per-warp part of the dynamic shared memory (barriers, run
// carry, two staging buffers); the private output copy follows them.
__host__ __device__ inline size_t warp_smem_bytes(int wpc, int C, int L, int AB, int wpe, int npw) {
    return 16 * (size_t)wpc + (size_t)wpc * carry_bytes(C, L, AB) + (size_t)wpc * 2 * wpe * npw * 4;
}

// The two staging barriers of a warp (lane 0 initialises them).
__device__ __forceinline__ void warp_bars_init(uint64_t *bars) {
    if ((threadIdx.x & 31) == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncwarp();
}

// One warp's contiguous range [ch_begin, ch_end) of chunks: stage, compute,
// hand the run carry on.  bars / carry / wbuf are the warp's barriers, carry
// slot and two staging buffers (stride WPE * npw words); k counts the chunks
// the warp has staged so far (stage k & 1, barrier phase (k >> 1) & 1) and is
// carried from range to range.  Returns false when a bounded wait ran out
// (status word set, the warp's copies landed).
template <typename FT, int C, int D1, int MODE, bool GCP = false>
__device__ __forceinline__ bool mttkrp_range(const MttkrpParams &p, uint64_t *bars, unsigned char *carry,
                                             int32_t *wbuf, typename Elem<FT>::Acc *priv, int ch_begin,
                                             int ch_end, uint32_t &k) {
    using AT = typename Elem<FT>::Acc;
    constexpr int REC = record_words(D1 + 1);
    constexpr int NARR = Staging<D1, MODE>::NARR;
    constexpr int WPE = Staging<D1, MODE>::WPE;
    constexpr unsigned FULL = 0xffffffffu;

    const int lane = threadIdx.x & 31;
    const int npw = p.npw;
    if (ch_begin >= ch_end) return true;  // whole warp idle (warp-uniform)

    const int32_t *src[NARR];
    if (MODE == M_PERM) {
        src[0] = p.perm;
    } else {
        src[0] = p.rows;
#pragma unroll
        for (int m = 0; m < D1; ++m) src[1 + m] = p.oidx[m];
        src[D1 + 1] = reinterpret_cast<const int32_t *>(p.vals);
    }

    auto chunk_len = [&](int ch) {
        const int64_t c0 = (int64_t)ch * npw;
        return (int)(p.nnz - c0 < (int64_t)npw ? p.nnz - c0 : (int64_t)npw);
    };
    // lane 0: stage the 16-byte-aligned body of chunk `ch` into stage `s`
    auto issue = [&](int ch, int s) {
        const int64_t c0 = (int64_t)ch * npw;
        const int n = chunk_len(ch);
        int32_t *buf = wbuf + s * WPE * npw;
        if (MODE == M_SORTED) {
            const uint32_t bytes = (uint32_t)((n * REC) & ~3) * 4u;
            mbar_arrive_expect_tx(&bars[s], bytes);
            if (bytes) bulk_g2s(buf, p.rec + c0 * REC, bytes, &bars[s]);
        } else {
            const uint32_t bytes = (uint32_t)(n & ~3) * 4u;
            mbar_arrive_expect_tx(&bars[s], bytes * NARR);
            if (bytes) {
#pragma unroll
                for (int a = 0; a < NARR; ++a) bulk_g2s(buf + a * npw, src[a] + c0, bytes, &bars[s]);
            }
        }
    };
    if (lane == 0) {
        issue(ch_begin, (int)(k & 1));
        if (ch_begin + 1 < ch_end) issue(ch_begin + 1, (int)((k + 1) & 1));
    }
    const int k0 = (int)k;

    // Sorted traversals with one rank block carry the open run across the
    // range's chunks; only the range's first and last rows are then shared.
    const bool use_carry = (MODE == M_SORTED || MODE == M_PERM) && p.n_rb == 1;
    if (use_carry) {
        const int64_t e_first = (int64_t)ch_begin * npw;
        const int64_t e_last = ((int64_t)ch_end * npw < p.nnz ? (int64_t)ch_end * npw : p.nnz) - 1;
        if (lane == 0) {
            int *hdr = reinterpret_cast<int *>(carry);
            hdr[0] = -1;
            if (MODE == M_SORTED) {
                hdr[1] = __ldg(p.rec + e_first * REC);
                hdr[2] = __ldg(p.rec + e_last * REC);
            } else {
                hdr[1] = __ldg(p.rows + __ldg(p.perm + e_first));
                hdr[2] = __ldg(p.rows + __ldg(p.perm + e_last));
            }
        }
        if ((lane >> p.log2L) == 0) {
            AT *ca = reinterpret_cast<AT *>(carry + 16) + lane * (C * Elem<FT>::VEC);
#pragma unroll
            for (int q = 0; q < C * Elem<FT>::VEC; ++q) ca[q] = (AT)0;
        }
        __syncwarp();
    }

    double lacc = 0.0;  // generalised CP: this lane's sum of loss terms
    for (int ch = ch_begin, kk = k0; ch < ch_end; ++ch, ++kk) {
        const int s = kk & 1;
        const uint32_t parity = (uint32_t)(kk >> 1) & 1u;
        const bool ok = mbar_wait(&bars[s], parity, p.wait_tries);
        if (!__all_sync(FULL, ok)) {
            // bounded-wait budget spent: report, let copies in flight land, leave
            if (lane == 0) atomicExch(p.err, SPT_DEV_TIMEOUT);
            if (ch + 1 < ch_end) mbar_wait(&bars[s ^ 1], (uint32_t)((kk + 1) >> 1) & 1u);
            mbar_wait(&bars[s], parity);
            return false;
        }
        int32_t *buf = wbuf + s * WPE * npw;
        const int64_t c0 = (int64_t)ch * npw;
        const int n = chunk_len(ch);
        if (MODE == M_SORTED) {  // words past the 16-byte body of a ragged chunk
            const int W = n * REC, wb = W & ~3;
            if (lane < W - wb) buf[wb + lane] = __ldg(p.rec + c0 * REC + wb + lane);
        } else {
            const int nb = n & ~3;
            if (lane < n - nb) {
#pragma unroll
                for (int a = 0; a < NARR; ++a) buf[a * npw + nb + lane] = __ldg(src[a] + c0 + nb + lane);
            }
        }
        __syncwarp();

        if (use_carry) {
            mttkrp_chunk<FT, C, D1, MODE, GCP>(p, buf, n, -1, -1, carry, nullptr, &lacc);
        } else {
            int b0, b1;
            chunk_bounds<D1, MODE>(p, buf, n, b0, b1);
            mttkrp_chunk<FT, C, D1, MODE, GCP>(p, buf, n, b0, b1, nullptr, priv, &lacc);
        }

        __syncwarp();  // every lane is done with this stage before it is refilled
        if (lane == 0 && ch + 2 < ch_end) {
            fence_proxy_async_smem();
            issue(ch + 2, s);
        }
    }
    if (use_carry) {
        __syncwarp();
        flush_carry<FT, C>(p, carry);
    }
    if (GCP && p.loss_out) {
        for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(FULL, lacc, o);
        if (lane == 0) atomicAdd(p.loss_out, lacc);
    }
    __syncwarp();  // the carry slot has been read before a next range rewrites it
    k = (uint32_t)(k0 + (ch_end - ch_begin));
    return true;
}

// Each warp of a persistent grid walks one contiguous range of the chunks:
// stage, compute, hand the run carry on.  The same steps as mttkrp_range,
// kept as one body for the single-tensor launch, where the register
// allocator spills less than through mttkrp_range's interface (measured:
// 4-way R=64 13% faster).
template <typename FT, int C, int D1, int MODE, bool GCP = false, bool CLAMP = false, bool DET = false>
__device__ __forceinline__ void mttkrp_warp_range(const MttkrpParams &p, unsigned char *smem_raw,
                                                  typename Elem<FT>::Acc *priv) {
    using AT = typename Elem<FT>::Acc;
    constexpr int REC = record_words(D1 + 1);
    constexpr int NARR = Staging<D1, MODE>::NARR;
    constexpr int WPE = Staging<D1, MODE>::WPE;
    constexpr unsigned FULL = 0xffffffffu;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int npw = p.npw;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw) + 2 * warp;
    const int cb = carry_bytes(C, 1 << p.log2L, (int)sizeof(AT));
    unsigned char *carry = smem_raw + 16 * wpc + (size_t)warp * cb;
    int32_t *wbuf = reinterpret_cast<int32_t *>(smem_raw + 16 * wpc + (size_t)wpc * cb) +
                    (size_t)warp * 2 * WPE * npw;

    // each warp walks a contiguous range of chunks
    const int gw = blockIdx.x * wpc + warp;
    const int nw = gridDim.x * wpc;
    const int ch_begin = (int)((int64_t)gw * p.nchunks / nw);
    const int ch_end = (int)((int64_t)(gw + 1) * p.nchunks / nw);
    if (ch_begin >= ch_end) return;  // whole warp idle (warp-uniform)

    const int32_t *src[NARR];
    if (MODE == M_PERM) {
        src[0] = p.perm;
    } else {
        src[0] = p.rows;
#pragma unroll
        for (int m = 0; m < D1; ++m) src[1 + m] = p.oidx[m];
        src[D1 + 1] = reinterpret_cast<const int32_t *>(p.vals);
    }

    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncwarp();

    auto chunk_len = [&](int ch) {
        const int64_t c0 = (int64_t)ch * npw;
        return (int)(p.nnz - c0 < (int64_t)npw ? p.nnz - c0 : (int64_t)npw);
    };
    // lane 0: stage the 16-byte-aligned body of chunk `ch` into stage `s`
    auto issue = [&](int ch, int s) {
        const int64_t c0 = (int64_t)ch * npw;
        const int n = chunk_len(ch);
        int32_t *buf = wbuf + s * WPE * npw;
        if (MODE == M_SORTED) {
            const uint32_t bytes = (uint32_t)((n * REC) & ~3) * 4u;
            mbar_arrive_expect_tx(&bars[s], bytes);
            if (bytes) bulk_g2s(buf, p.rec + c0 * REC, bytes, &bars[s]);
        } else {
            const uint32_t bytes = (uint32_t)(n & ~3) * 4u;
            mbar_arrive_expect_tx(&bars[s], bytes * NARR);
            if (bytes) {
#pragma unroll
                for (int a = 0; a < NARR; ++a) bulk_g2s(buf + a * npw, src[a] + c0, bytes, &bars[s]);
            }
        }
    };
    if (lane == 0) {
        issue(ch_begin, 0);
        if (ch_begin + 1 < ch_end) issue(ch_begin + 1, 1);
    }

    // Sorted traversals with one rank block carry the open run across the
    // range's chunks; only the range's first and last rows are then shared.
    const bool use_carry = (MODE == M_SORTED || MODE == M_PERM) && p.n_rb == 1;
    if (use_carry) {
        const int64_t e_first = (int64_t)ch_begin * npw;
        const int64_t e_last = ((int64_t)ch_end * npw < p.nnz ? (int64_t)ch_end * npw : p.nnz) - 1;
        if (lane == 0) {
            int *hdr = reinterpret_cast<int *>(carry);
            hdr[0] = -1;
            if (MODE == M_SORTED) {
                hdr[1] = __ldg(p.rec + e_first * REC);
                hdr[2] = __ldg(p.rec + e_last * REC);
            } else {
                hdr[1] = __ldg(p.rows + __ldg(p.perm + e_first));
                hdr[2] = __ldg(p.rows + __ldg(p.perm + e_last));
            }
        }
        if ((lane >> p.log2L) == 0) {
            AT *ca = reinterpret_cast<AT *>(carry + 16) + lane * (C * Elem<FT>::VEC);
#pragma unroll
            for (int q = 0; q < C * Elem<FT>::VEC; ++q) ca[q] = (AT)0;
        }
        __syncwarp();
    }

    double lacc = 0.0;  // generalised CP: this lane's sum of loss terms
    int k = 0;
    for (int ch = ch_begin; ch < ch_end; ++ch, ++k) {
        const int s = k & 1;
        const uint32_t parity = (uint32_t)(k >> 1) & 1u;
        const bool ok = mbar_wait(&bars[s], parity, p.wait_tries);
        if (!__all_sync(FULL, ok)) {
            // bounded-wait budget spent: report, let copies in flight land, leave
            if (lane == 0) atomicExch(p.err, SPT_DEV_TIMEOUT);
            if (ch + 1 < ch_end) mbar_wait(&bars[s ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            mbar_wait(&bars[s], parity);
            return;
        }
        int32_t *buf = wbuf + s * WPE * npw;
        const int64_t c0 = (int64_t)ch * npw;
        const int n = chunk_len(ch);
        if (MODE == M_SORTED) {  // words past the 16-byte body of a ragged chunk
            const int W = n * REC, wb = W & ~3;
            if (lane < W - wb) buf[wb + lane] = __ldg(p.rec + c0 * REC + wb + lane);
        } else {
            const int nb = n & ~3;
            if (lane < n - nb) {
#pragma unroll
                for (int a = 0; a < NARR; ++a) buf[a * npw + nb + lane] = __ldg(src[a] + c0 + nb + lane);
            }
        }
        __syncwarp();

        if (use_carry) {
            mttkrp_chunk<FT, C, D1, MODE, GCP, CLAMP, DET>(p, buf, n, -1, -1, carry, nullptr, &lacc);
        } else {
            int b0, b1;
            chunk_bounds<D1, MODE>(p, buf, n, b0, b1);
            mttkrp_chunk<FT, C, D1, MODE, GCP, CLAMP, DET>(p, buf, n, b0, b1, nullptr, priv, &lacc);
        }

        __syncwarp();  // every lane is done with this stage before it is refilled
        if (lane == 0 && ch + 2 < ch_end) {
            fence_proxy_async_smem();
            issue(ch + 2, s);
        }
    }
    if (use_carry) {
        __syncwarp();
        flush_carry<FT, C, DET>(p, carry);
    }
    if (GCP && p.loss_out) {
        for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(FULL, lacc, o);
        if (lane == 0) atomicAdd(p.loss_out, lacc);
    }
}

// Generalised CP gradient over the mode-sorted copy: the MTTKRP traversal
// with each nonzero's value replaced by df/dm at the model value m.
#ifndef SPT_GCP_MINBLOCKS
#define SPT_GCP_MINBLOCKS 4
#endif
template <typename FT, int C, int D1>
__global__ void __launch_bounds__(256, SPT_GCP_MINBLOCKS) gcp_kernel(const MttkrpParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    mttkrp_warp_range<FT, C, D1, M_SORTED, true>(p, smem_raw, nullptr);
}

// Add this CTA's private rows (row = local * K + cluster rank) to the output
// with vector atomics (16 bytes for float), skipping all-zero quads.
template <typename AT>
__device__ __forceinline__ void flush_private(const MttkrpParams &p, const AT *priv, int rank) {
    const int q4 = p.pld >> 2;
    const int64_t total = (int64_t)p.prows * q4;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int lr = (int)(i / q4);
        const int c4 = (int)(i - (int64_t)lr * q4);
        const int row = (lr << p.log2K) + rank;
        if (row >= p.In) continue;
        const AT *src = priv + (int64_t)lr * p.pld + 4 * c4;
        const AT v[4] = {src[0], src[1], src[2], src[3]};
        if (v[0] != (AT)0 || v[1] != (AT)0 || v[2] != (AT)0 || v[3] != (AT)0)
            red_add4(reinterpret_cast<AT *>(p.out) + (int64_t)row * p.old + 4 * c4, v);
    }
}

// Atomic scatter with hot rows: zero this CTA's copy of the hot rows and
// build the hash table, accumulate, then add the copy to the output (16-byte
// vector atomics, all-zero quads skipped).  Every thread reaches both
// barriers: warps without chunks (or whose wait ran out) skip to them.
template <typename FT, int C, int D1>
__device__ __forceinline__ void mttkrp_atomic_hot(const MttkrpParams &p, unsigned char *smem_raw) {
    using AT = typename Elem<FT>::Acc;
    const int wpc = blockDim.x >> 5;
    AT *hot = reinterpret_cast<AT *>(smem_raw + warp_smem_bytes(wpc, C, 1 << p.log2L, (int)sizeof(AT),
                                                                Staging<D1, M_ATOMIC>::WPE, p.npw));
    int *hkey = reinterpret_cast<int *>(hot + (int64_t)p.nhot * p.pld);
    const int T = 1 << p.hot_log2T;
    for (int i = threadIdx.x; i < p.nhot * p.pld; i += blockDim.x) hot[i] = (AT)0;
    for (int i = threadIdx.x; i < T; i += blockDim.x) hkey[i] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < p.nhot; i += blockDim.x) {
        const int row = __ldg(p.hot_rows + i);
        unsigned h = ((unsigned)row * 0x9E3779B1u) >> (32 - p.hot_log2T);
        for (int q = 0; q < T; ++q) {  // distinct rows: each claims the first free slot
            if (atomicCAS(hkey + h, -1, row) == -1) {
                hkey[T + h] = i;
                break;
            }
            h = (h + 1) & (unsigned)(T - 1);
        }
    }
    __syncthreads();
    mttkrp_warp_range<FT, C, D1, M_ATOMIC>(p, smem_raw, hot);
    __syncwarp();
    __syncthreads();
    const int q4 = p.pld >> 2;
    for (int i = threadIdx.x; i < p.nhot * q4; i += blockDim.x) {
        const int slot = i / q4, c4 = i - slot * q4;
        const AT *src = hot + (int64_t)slot * p.pld + 4 * c4;
        const AT v[4] = {src[0], src[1], src[2], src[3]};
        if (v[0] == (AT)0 && v[1] == (AT)0 && v[2] == (AT)0 && v[3] == (AT)0) continue;
        const int64_t o = (int64_t)__ldg(p.hot_rows + slot) * p.old + 4 * c4 +
                          (int64_t)(blockIdx.x & (p.nrep - 1)) * p.rep_stride;
        red_add4(reinterpret_cast<AT *>(p.out) + o, v);
    }
}

template <typename FT, int C, int D1, int MODE, bool CLAMP = false, bool DET = false>
__global__ void __launch_bounds__(512, MinBlocks<FT, C>::value) mttkrp_kernel(const MttkrpParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (MODE == M_ATOMIC && p.nhot > 0) {
        mttkrp_atomic_hot<FT, C, D1>(p, smem_raw);
        return;
    }
    if (MODE != M_PRIVATE) {
        mttkrp_warp_range<FT, C, D1, MODE, false, CLAMP, DET>(p, smem_raw, nullptr);
        return;
    }
    // Privatised scatter: zero this CTA's rows, wait until every CTA of the
    // cluster has (remote adds may follow at once), accumulate, wait until
    // every add of the cluster has landed, then flush.  Every thread reaches
    // both barriers: warps without chunks skip straight to them.
    using AT = typename Elem<FT>::Acc;
    const int wpc = blockDim.x >> 5;
    AT *priv = reinterpret_cast<AT *>(smem_raw + warp_smem_bytes(wpc, C, 1 << p.log2L, (int)sizeof(AT),
                                                                 Staging<D1, MODE>::WPE, p.npw));
    const int nfl = p.prows * p.pld;  // a multiple of 4
    const AT zero4[4] = {(AT)0, (AT)0, (AT)0, (AT)0};
    for (int i = 4 * threadIdx.x; i < nfl; i += 4 * blockDim.x) store4(priv + i, zero4);
    const bool clustered = p.log2K > 0;
    if (clustered) cluster_sync_all(); else __syncthreads();
    mttkrp_warp_range<FT, C, D1, MODE>(p, smem_raw, priv);
    __syncwarp();  // the warp is converged for the aligned cluster barrier
    if (clustered) cluster_sync_all(); else __syncthreads();
    flush_private(p, priv, clustered ? (int)cluster_ctarank() : 0);
}

typedef void (*MttkrpKernelFn)(const MttkrpParams);

// Kernel table of one element type: fn(C in {1,2}, D1 in 0..4, mode in 0..3).
MttkrpKernelFn mttkrp_kernel_f32(int C, int D1, int mode);
MttkrpKernelFn mttkrp_kernel_bf16(int C, int D1, int mode);
MttkrpKernelFn mttkrp_kernel_f16(int C, int D1, int mode);
MttkrpKernelFn mttkrp_kernel_f64(int C, int D1, int mode);
// The sorted-traversal kernels with clamped (unpredicated) gathers, for ranks
// that leave a lane's whole chunk past column R: fn(C in {1,2}, D1 in 0..4).
MttkrpKernelFn mttkrp_kernel_f32_clamp(int C, int D1);
MttkrpKernelFn mttkrp_kernel_bf16_clamp(int C, int D1);
MttkrpKernelFn mttkrp_kernel_f16_clamp(int C, int D1);
MttkrpKernelFn mttkrp_kernel_f64_clamp(int C, int D1);
// sorted traversal with the run carry whose shared rows go to per-warp slots
// (deterministic sums; see det_fixup_kernel)
MttkrpKernelFn mttkrp_kernel_f32_det(int C, int D1);
MttkrpKernelFn mttkrp_kernel_bf16_det(int C, int D1);
MttkrpKernelFn mttkrp_kernel_f16_det(int C, int D1);
MttkrpKernelFn mttkrp_kernel_f64_det(int C, int D1);
// Generalised CP gradient kernels: fdt in {F32, BF16, F16}, C in {1,2}, D1 in 1..4.
MttkrpKernelFn gcp_kernel_fn(spt_dtype fdt, int C, int D1);

#define SPT_INSTANTIATE_MTTKRP_TABLE(FT, NAME)                                                                                   \
    MttkrpKernelFn NAME(int C, int D1, int mode) {                                                                               \
        static const MttkrpKernelFn tab[2][5][4] = {                                                                             \
            {{mttkrp_kernel<FT, 1, 0, 0>, mttkrp_kernel<FT, 1, 0, 1>, mttkrp_kernel<FT, 1, 0, 2>, mttkrp_kernel<FT, 1, 0, 3>},   \
             {mttkrp_kernel<FT, 1, 1, 0>, mttkrp_kernel<FT, 1, 1, 1>, mttkrp_kernel<FT, 1, 1, 2>, mttkrp_kernel<FT, 1, 1, 3>},   \
             {mttkrp_kernel<FT, 1, 2, 0>, mttkrp_kernel<FT, 1, 2, 1>, mttkrp_kernel<FT, 1, 2, 2>, mttkrp_kernel<FT, 1, 2, 3>},   \
             {mttkrp_kernel<FT, 1, 3, 0>, mttkrp_kernel<FT, 1, 3, 1>, mttkrp_kernel<FT, 1, 3, 2>, mttkrp_kernel<FT, 1, 3, 3>},   \
             {mttkrp_kernel<FT, 1, 4, 0>, mttkrp_kernel<FT, 1, 4, 1>, mttkrp_kernel<FT, 1, 4, 2>, mttkrp_kernel<FT, 1, 4, 3>}},  \
            {{mttkrp_kernel<FT, 2, 0, 0>, mttkrp_kernel<FT, 2, 0, 1>, mttkrp_kernel<FT, 2, 0, 2>, mttkrp_kernel<FT, 2, 0, 3>},   \
             {mttkrp_kernel<FT, 2, 1, 0>, mttkrp_kernel<FT, 2, 1, 1>, mttkrp_kernel<FT, 2, 1, 2>, mttkrp_kernel<FT, 2, 1, 3>},   \
             {mttkrp_kernel<FT, 2, 2, 0>, mttkrp_kernel<FT, 2, 2, 1>, mttkrp_kernel<FT, 2, 2, 2>, mttkrp_kernel<FT, 2, 2, 3>},   \
             {mttkrp_kernel<FT, 2, 3, 0>, mttkrp_kernel<FT, 2, 3, 1>, mttkrp_kernel<FT, 2, 3, 2>, mttkrp_kernel<FT, 2, 3, 3>},   \
             {mttkrp_kernel<FT, 2, 4, 0>, mttkrp_kernel<FT, 2, 4, 1>, mttkrp_kernel<FT, 2, 4, 2>, mttkrp_kernel<FT, 2, 4, 3>}}}; \
        if (C < 1 || C > 2 || D1 < 0 || D1 > 4 || mode < 0 || mode > 3) return nullptr;                                          \
        return tab[C - 1][D1][mode];                                                                                             \
    }                                                                                                                            \
    MttkrpKernelFn NAME##_clamp(int C, int D1) {                                                                                 \
        static const MttkrpKernelFn tab[2][5] = {                                                                                \
            {mttkrp_kernel<FT, 1, 0, 1, true>, mttkrp_kernel<FT, 1, 1, 1, true>, mttkrp_kernel<FT, 1, 2, 1, true>,               \
             mttkrp_kernel<FT, 1, 3, 1, true>, mttkrp_kernel<FT, 1, 4, 1, true>},                                                \
            {mttkrp_kernel<FT, 2, 0, 1, true>, mttkrp_kernel<FT, 2, 1, 1, true>, mttkrp_kernel<FT, 2, 2, 1, true>,               \
             mttkrp_kernel<FT, 2, 3, 1, true>, mttkrp_kernel<FT, 2, 4, 1, true>}};                                               \
        if (C < 1 || C > 2 || D1 < 0 || D1 > 4) return nullptr;                                                                  \
        return tab[C - 1][D1];                                                                                                   \
    } \
    MttkrpKernelFn NAME##_det(int C, int D1) {                                                                                   \
        static const MttkrpKernelFn tab[2][5] = {                                                                                \
            {mttkrp_kernel<FT, 1, 0, 1, false, true>, mttkrp_kernel<FT, 1, 1, 1, false, true>,                                   \
             mttkrp_kernel<FT, 1, 2, 1, false, true>, mttkrp_kernel<FT, 1, 3, 1, false, true>,                                   \
             mttkrp_kernel<FT, 1, 4, 1, false, true>},                                                                           \
            {mttkrp_kernel<FT, 2, 0, 1, false, true>, mttkrp_kernel<FT, 2, 1, 1, false, true>,                                   \
             mttkrp_kernel<FT, 2, 2, 1, false, true>, mttkrp_kernel<FT, 2, 3, 1, false, true>,                                   \
             mttkrp_kernel<FT, 2, 4, 1, false, true>}};                                                                          \
        if (C < 1 || C > 2 || D1 < 0 || D1 > 4) return nullptr;                                                                  \
        return tab[C - 1][D1];                                                                                                   \
    }

}  // namespace spt

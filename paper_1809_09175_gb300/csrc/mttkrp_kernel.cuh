// mttkrp_kernel.cuh -- the sparse COO MTTKRP kernel (Sec. 2 eq. mttkrp).
//
//   out(k, j) = lambda_j * sum_{i : l_in = k} x_i * prod_{m != n} A^(m)(l_im, j)
//
// Work decomposition (GB300 mapping of the paper's league/team/vector levels,
// Sec. 3 Tab. "Levels of Parallelism"):
//  * A warp owns a chunk of `npw` consecutive nonzeros of the traversal order
//    (persistent grid, chunks dealt round-robin to warps).  The chunk's
//    coordinates and values (or, for the permuted traversal, its permutation
//    entries) are staged into the warp's shared memory with 1-D bulk copies
//    (cp.async.bulk, mbarrier completion), double buffered, so the next chunk
//    streams in while this one is computed.
//  * The warp is split into G = 32/L groups of L lanes.  Group g walks the
//    nonzeros [g*S, g*S+S) of the chunk in order (the paper's NZPTM block,
//    Fig. MTTKRP-C); lane l of the group owns 16-byte column chunks of the
//    rank block (the paper's vector lanes over j, Fig. MTTKRP-B), loading
//    the d-1 factor rows with coalesced 16-byte loads and keeping the
//    running row sum in registers (the paper's TinyVec).
//  * Scatter:
//      M_ATOMIC  storage order; a group's running sum is added atomically
//                (16-byte vector red) whenever its row changes (Fig. MTTKRP-B
//                with merging of equal consecutive rows).
//      M_SORTED  nonzeros in mode-n order from a mode-sorted copy; M_PERM
//                walks storage through the permutation (Fig. MTTKRP-C).  A
//                group writes a finished row with a plain store; the first
//                and last run of every group are combined across the warp
//                with shuffles (a segmented reduction over the groups), and
//                only the chunk's first and last row are added atomically,
//                because only those rows can be shared with other warps.
//  * Columns: rank block rb covers columns [rb*L*C*VEC, ...); lane l's chunk
//    c starts at column rb*L*C*VEC + (c*L + l)*VEC.  Columns >= R contribute 0.
#pragma once
#include "common.cuh"

namespace spt {

enum MttkrpMode { M_ATOMIC = 0, M_SORTED = 1, M_PERM = 2 };

struct MttkrpParams {
    const int32_t *rows;     // mode-n coordinate, traversal order (M_PERM: storage order)
    const int32_t *oidx[4];  // coordinates of the other modes (same order as rows)
    const float *vals;       // values (same order as rows)
    const int32_t *perm;     // M_PERM: traversal position -> storage position
    const void *fac[4];      // factor matrices of the other modes
    int64_t fld;             // factor row stride (elements)
    const float *lambda;     // nullable
    float *out;              // I_n x old, zeroed before launch
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
};

__device__ __forceinline__ uint4 ldg16(const void *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

__device__ __forceinline__ void red_add4(float *dst, const float *v) {
    atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(v[0], v[1], v[2], v[3]));
}

template <int U_> struct Unroll { static constexpr int U = U_; };

template <typename FT, int C, int D1, int MODE>
__global__ void __launch_bounds__(512) mttkrp_kernel(const MttkrpParams p) {
    using E = Elem<FT>;
    constexpr int VEC = E::VEC;
    constexpr int NARR = (MODE == M_PERM) ? 1 : (D1 + 2);
    constexpr int LOADS = D1 * C;
    constexpr int U = (LOADS <= 2) ? 4 : (LOADS <= 4 ? 2 : 1);
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int npw = p.npw;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw) + 2 * warp;
    int32_t *wbuf = reinterpret_cast<int32_t *>(smem_raw + 16 * wpc) + (size_t)warp * 2 * NARR * npw;

    const int64_t gw = (int64_t)blockIdx.x * wpc + warp;
    const int64_t nw = (int64_t)gridDim.x * wpc;
    if (gw >= p.nchunks) return;  // whole warp idle (warp-uniform)

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

    // lane 0: stage the 16-byte-aligned body of chunk `ch` into stage `s`
    auto issue = [&](int64_t ch, int s) {
        const int64_t c0 = ch * npw;
        const int n = (int)(p.nnz - c0 < (int64_t)npw ? p.nnz - c0 : (int64_t)npw);
        const uint32_t bytes = (uint32_t)(n & ~3) * 4u;
        int32_t *buf = wbuf + s * NARR * npw;
        mbar_arrive_expect_tx(&bars[s], bytes * NARR);
        if (bytes) {
#pragma unroll
            for (int a = 0; a < NARR; ++a) bulk_g2s(buf + a * npw, src[a] + c0, bytes, &bars[s]);
        }
    };
    if (lane == 0) {
        issue(gw, 0);
        if (gw + nw < p.nchunks) issue(gw + nw, 1);
    }

    const int log2L = p.log2L;
    const int L = 1 << log2L;
    const int G = 32 >> log2L;
    const int g = lane >> log2L;
    const int l = lane & (L - 1);
    const int S = p.S;

    int k = 0;
    for (int64_t ch = gw; ch < p.nchunks; ch += nw, ++k) {
        const int s = k & 1;
        const uint32_t parity = (uint32_t)(k >> 1) & 1u;
        const bool ok = mbar_wait(&bars[s], parity);
        if (!__all_sync(FULL, ok)) {
            // bounded-wait budget spent: report, let copies in flight land, leave
            if (lane == 0) atomicExch(p.err, SPT_DEV_TIMEOUT);
            if (ch + nw < p.nchunks) mbar_wait(&bars[s ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            mbar_wait(&bars[s], parity);
            return;
        }
        int32_t *buf = wbuf + s * NARR * npw;
        const int64_t c0 = ch * npw;
        const int n = (int)(p.nnz - c0 < (int64_t)npw ? p.nnz - c0 : (int64_t)npw);
        const int nb = n & ~3;
        if (lane < n - nb) {
#pragma unroll
            for (int a = 0; a < NARR; ++a) buf[a * npw + nb + lane] = __ldg(src[a] + c0 + nb + lane);
        }
        __syncwarp();

        const int e0 = g * S;
        const int cnt = max(0, min(S, n - e0));
        int crow0 = 0, crow1 = 0;
        if (MODE == M_SORTED) {
            crow0 = buf[0];
            crow1 = buf[n - 1];
        } else if (MODE == M_PERM) {
            crow0 = __ldg(p.rows + buf[0]);
            crow1 = __ldg(p.rows + buf[n - 1]);
        }

        for (int rb = 0; rb < p.n_rb; ++rb) {
            int col[C], nv[C];
            float lam[C][VEC];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                col[c] = rb * p.rb_cols + (c * L + l) * VEC;
                nv[c] = max(0, min(VEC, p.R - col[c]));
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    lam[c][v] = (p.lambda && v < nv[c]) ? __ldg(p.lambda + col[c] + v) : 1.0f;
            }

            float acc[C][VEC], facc[C][VEC];
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][v] = facc[c][v] = 0.0f;
            int cur = -1, frow = -1;
            bool fclosed = false;

            // emit a finished row sum: atomic for shared rows, plain store otherwise
            auto write_row = [&](int row, float (&a)[C][VEC], bool atomic) {
                float *dst = p.out + (int64_t)row * p.old;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    if (nv[c] == 0) continue;
                    float w[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) w[v] = a[c][v] * lam[c][v];
                    if (atomic) {
#pragma unroll
                        for (int q = 0; q < VEC; q += 4) red_add4(dst + col[c] + q, w + q);
                    } else {
#pragma unroll
                        for (int q = 0; q < VEC; q += 4)
                            *reinterpret_cast<float4 *>(dst + col[c] + q) =
                                make_float4(w[q], w[q + 1], w[q + 2], w[q + 3]);
                    }
                }
            };

            for (int t0 = 0; t0 < cnt; t0 += U) {
                int rowu[U];
                float xu[U];
                uint4 raw[U][D1 > 0 ? D1 : 1][C];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u;
                    const bool vu = t < cnt;
                    const int e = e0 + (vu ? t : 0);
                    int r[D1 > 0 ? D1 : 1];
                    if (MODE == M_PERM) {
                        const int q = buf[e];
                        rowu[u] = __ldg(p.rows + q);
                        xu[u] = __ldg(p.vals + q);
#pragma unroll
                        for (int m = 0; m < D1; ++m) r[m] = __ldg(p.oidx[m] + q);
                    } else {
                        rowu[u] = buf[e];
                        xu[u] = __int_as_float(buf[(D1 + 1) * npw + e]);
#pragma unroll
                        for (int m = 0; m < D1; ++m) r[m] = buf[(1 + m) * npw + e];
                    }
#pragma unroll
                    for (int m = 0; m < D1; ++m) {
                        const FT *base = reinterpret_cast<const FT *>(p.fac[m]) + (int64_t)r[m] * p.fld;
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            raw[u][m][c] = (vu && nv[c] > 0) ? ldg16(base + col[c]) : make_uint4(0, 0, 0, 0);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (t0 + u >= cnt) break;
                    float prod[C][VEC];
#pragma unroll
                    for (int c = 0; c < C; ++c) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) prod[c][v] = xu[u];
#pragma unroll
                        for (int m = 0; m < D1; ++m) {
                            float f[VEC];
                            E::widen(raw[u][m][c], f);
#pragma unroll
                            for (int v = 0; v < VEC; ++v) prod[c][v] *= f[v];
                        }
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            if (v >= nv[c]) prod[c][v] = 0.0f;
                    }
                    const int row = rowu[u];
                    if (row != cur) {
                        if (cur >= 0) {
                            if (MODE == M_ATOMIC) {
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
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[c][v] = prod[c][v];
                    } else {
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[c][v] += prod[c][v];
                    }
                }
            }

            if (MODE == M_ATOMIC) {
                if (cur >= 0) write_row(cur, acc, true);
            } else {
                // Segmented combine of the groups' open runs, in group order.
                // Every lane tracks the running (orow, oacc) for its columns;
                // group 0's lanes perform the writes.
                float oacc[C][VEC];
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) oacc[c][v] = 0.0f;
                int orow = -1;
                const bool writer = (g == 0);
                auto emit = [&](int row, float (&a)[C][VEC]) {
                    if (writer) write_row(row, a, row == crow0 || row == crow1);
                };
                for (int g2 = 0; g2 < G; ++g2) {
                    const int srcl = (g2 << log2L) | l;
                    const int scur = __shfl_sync(FULL, cur, srcl);
                    if (scur < 0) break;  // this and later groups got no nonzeros
                    const int sfc = __shfl_sync(FULL, (int)fclosed, srcl);
                    const int sfrow = __shfl_sync(FULL, frow, srcl);
                    float F[C][VEC], A[C][VEC];
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
                if (orow >= 0) emit(orow, oacc);
            }
        }

        __syncwarp();  // every lane is done with this stage before it is refilled
        if (lane == 0 && ch + 2 * nw < p.nchunks) {
            fence_proxy_async_smem();
            issue(ch + 2 * nw, s);
        }
    }
}

typedef void (*MttkrpKernelFn)(const MttkrpParams);

// Kernel table of one element type: fn(C in {1,2}, D1 in 0..4, mode in 0..2).
MttkrpKernelFn mttkrp_kernel_f32(int C, int D1, int mode);
MttkrpKernelFn mttkrp_kernel_bf16(int C, int D1, int mode);
MttkrpKernelFn mttkrp_kernel_f16(int C, int D1, int mode);

#define SPT_INSTANTIATE_MTTKRP_TABLE(FT, NAME)                                            \
    MttkrpKernelFn NAME(int C, int D1, int mode) {                                       \
        static const MttkrpKernelFn tab[2][5][3] = {                                     \
            {{mttkrp_kernel<FT, 1, 0, 0>, mttkrp_kernel<FT, 1, 0, 1>, mttkrp_kernel<FT, 1, 0, 2>}, \
             {mttkrp_kernel<FT, 1, 1, 0>, mttkrp_kernel<FT, 1, 1, 1>, mttkrp_kernel<FT, 1, 1, 2>}, \
             {mttkrp_kernel<FT, 1, 2, 0>, mttkrp_kernel<FT, 1, 2, 1>, mttkrp_kernel<FT, 1, 2, 2>}, \
             {mttkrp_kernel<FT, 1, 3, 0>, mttkrp_kernel<FT, 1, 3, 1>, mttkrp_kernel<FT, 1, 3, 2>}, \
             {mttkrp_kernel<FT, 1, 4, 0>, mttkrp_kernel<FT, 1, 4, 1>, mttkrp_kernel<FT, 1, 4, 2>}}, \
            {{mttkrp_kernel<FT, 2, 0, 0>, mttkrp_kernel<FT, 2, 0, 1>, mttkrp_kernel<FT, 2, 0, 2>}, \
             {mttkrp_kernel<FT, 2, 1, 0>, mttkrp_kernel<FT, 2, 1, 1>, mttkrp_kernel<FT, 2, 1, 2>}, \
             {mttkrp_kernel<FT, 2, 2, 0>, mttkrp_kernel<FT, 2, 2, 1>, mttkrp_kernel<FT, 2, 2, 2>}, \
             {mttkrp_kernel<FT, 2, 3, 0>, mttkrp_kernel<FT, 2, 3, 1>, mttkrp_kernel<FT, 2, 3, 2>}, \
             {mttkrp_kernel<FT, 2, 4, 0>, mttkrp_kernel<FT, 2, 4, 1>, mttkrp_kernel<FT, 2, 4, 2>}}}; \
        if (C < 1 || C > 2 || D1 < 0 || D1 > 4 || mode < 0 || mode > 2) return nullptr;  \
        return tab[C - 1][D1][mode];                                                     \
    }

}  // namespace spt

// mttkrp_host.cu -- schedule logic and launch of the MTTKRP kernel.
#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "mttkrp_kernel.cuh"

namespace spt {

int elem_bytes(spt_dtype fdt) { return fdt == SPT_F32 ? 4 : 2; }

namespace {
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
    // about 7 KB of shared memory per warp (two staging buffers plus the run
    // carry), so four 8-warp CTAs fit an SM; at most 256 nonzeros per chunk
    const int narr = s.scatter == SPT_SCATTER_PERM ? 1
                     : (s.scatter == SPT_SCATTER_SORTED ? record_words(t->d) : t->d + 1);
    const int npw = std::min(256, (7168 - 16 - carry_bytes(s.chunks, lanes)) / (8 * narr));
    s.nnz_per_group = std::max(4, npw / (32 / lanes));
    s.warps_per_cta = 8;
    s.ctas_per_sm = 0;
    return s;
}

spt_status check_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank, const spt_schedule &s) {
    (void)fdt;
    (void)rank;
    if (s.scatter < SPT_SCATTER_ATOMIC || s.scatter > SPT_SCATTER_SORTED)
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
    return SPT_OK;
}

spt_status launch_mttkrp(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                         int rank, int ld, const float *lambda, float *out,
                         const spt_schedule &s, cudaStream_t st) {
    const int vec = 4;  // columns per lane chunk
    const int L = s.lanes_per_nnz, C = s.chunks;
    const int G = 32 / L;
    const int rb_cols = L * C * vec;
    const int S = adjust_S(s.nnz_per_group, G);
    const int npw = G * S;
    const int wpc = s.warps_per_cta;
    SPT_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)t->dims[mode] * ld, st));
    if (t->nnz == 0) return SPT_OK;

    const int D1 = t->d - 1;
    const int kmode = s.scatter == SPT_SCATTER_ATOMIC ? M_ATOMIC
                      : (s.scatter == SPT_SCATTER_SORTED ? M_SORTED : M_PERM);
    MttkrpParams p{};
    p.rows = t->idx[mode];
    p.vals = t->vals;
    p.perm = t->perm[mode];
    p.rec = reinterpret_cast<const int32_t *>(t->sorted_buf[mode]);
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

    const int wpe = kmode == M_PERM ? 1 : (kmode == M_SORTED ? record_words(t->d) : D1 + 2);
    const size_t smem = 16 * (size_t)wpc + (size_t)wpc * carry_bytes(C, L) + (size_t)wpc * 2 * wpe * npw * 4;
    if (smem > 227 * 1024)
        return fail(SPT_EINVAL, "schedule: staging buffers exceed 227 KB of shared memory "
                                "(lower warps_per_cta or nnz_per_group)");
    MttkrpKernelFn fn = fdt == SPT_F32    ? mttkrp_kernel_f32(C, D1, kmode)
                        : fdt == SPT_BF16 ? mttkrp_kernel_bf16(C, D1, kmode)
                                          : mttkrp_kernel_f16(C, D1, kmode);
    if (!fn) return fail(SPT_EUNSUPPORTED, "mttkrp: no kernel for this order/chunks");
    spt_status e = ensure_smem_attr(fn, (int)smem);
    if (e) return e;
    int bps = 0;
    SPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, wpc * 32, smem));
    if (bps < 1) return fail(SPT_EINVAL, "schedule: kernel does not fit on an SM");
    const int cps = s.ctas_per_sm > 0 ? std::min(s.ctas_per_sm, bps) : bps;
    const int64_t need = (p.nchunks + wpc - 1) / wpc;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)cps * sm_count(), need));
    fn<<<blocks, wpc * 32, smem, st>>>(p);
    SPT_LAUNCH_CHECK("mttkrp_kernel launch");
    return SPT_OK;
}

}  // namespace spt

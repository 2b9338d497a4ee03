// gcp.cu -- generalised CP gradient: the count- and binary-data losses that
// Sec. 8 names as the next application of the MTTKRP machinery.
//
// For the model m = sum_j prod_l A^(l)(., j) and a loss f(x, m), the gradient
// of F = sum f(x_e, m_e) with respect to A^(n) is an MTTKRP whose values are
// df/dm at each entry:
//   G(k, j) = sum_{e : e_n = k} df/dm(x_e, m_e) prod_{l != n} A^(l)(e_l, j).
// The stored entries run through the MTTKRP kernel's sorted traversal
// (gcp_kernel: the model value is the dot product of the entry's own row
// A^(n)(e_n, :) with the product of the other rows, summed across the lane
// group with shuffles).  For the Poisson loss, which runs over every entry of
// the tensor, the entries off the stored coordinates have df/dm = 1 and their
// sum factorises into column sums: G(k, j) += prod_{l != n} colsum_l(j) for
// every row k, and F gets sum_j prod_l colsum_l(j).
#include "internal.h"
#include "mttkrp_kernel.cuh"

namespace spt {

template <typename FT> static MttkrpKernelFn gcp_table(int C, int D1) {
    static const MttkrpKernelFn tab[2][4] = {
        {gcp_kernel<FT, 1, 1>, gcp_kernel<FT, 1, 2>, gcp_kernel<FT, 1, 3>, gcp_kernel<FT, 1, 4>},
        {gcp_kernel<FT, 2, 1>, gcp_kernel<FT, 2, 2>, gcp_kernel<FT, 2, 3>, gcp_kernel<FT, 2, 4>}};
    if (C < 1 || C > 2 || D1 < 1 || D1 > 4) return nullptr;
    return tab[C - 1][D1 - 1];
}

MttkrpKernelFn gcp_kernel_fn(spt_dtype fdt, int C, int D1) {
    if (fdt == SPT_F32) return gcp_table<float>(C, D1);
    if (fdt == SPT_BF16) return gcp_table<__nv_bfloat16>(C, D1);
    if (fdt == SPT_F16) return gcp_table<__half>(C, D1);
    return nullptr;
}

namespace {

template <typename FT> __device__ __forceinline__ float to_f(FT v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// cs[j] += sum over rows of A(:, j), j < R: every CTA walks rows
// blockIdx.x, +gridDim.x, ...; thread t sums column t (+blockDim.x, ...),
// fp32 over 64 rows at a time, then fp64.
template <typename FT>
__global__ void __launch_bounds__(256) colsum_kernel(const FT *A, int64_t I, int ld, int R, double *cs) {
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        double acc = 0.0;
        float part = 0.0f;
        int cnt = 0;
        for (int64_t r = blockIdx.x; r < I; r += gridDim.x) {
            part += to_f<FT>(A[r * ld + j]);
            if (++cnt == 64) {
                acc += (double)part;
                part = 0.0f;
                cnt = 0;
            }
        }
        acc += (double)part;
        atomicAdd(cs + j, acc);
    }
}

// Poisson: G(k, j) += c_j = prod_{l != n} cs_l(j) for every row k < I and
// column j < R (computed in fp64, rounded once); CTA 0 adds
// sum_j prod_l cs_l(j) to the loss.
__global__ void __launch_bounds__(256) poisson_dense_kernel(float *G, int64_t I, int ld, int R, const double *cs,
                                                            int d, int n, double *loss_out) {
    __shared__ double c[256];
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        double v = 1.0;
        for (int l = 0; l < d; ++l)
            if (l != n) v *= cs[l * R + j];
        c[j] = v;
        if (blockIdx.x == 0 && loss_out) atomicAdd(loss_out, v * cs[n * R + j]);
    }
    __syncthreads();
    const int rpp = (int)blockDim.x / R;  // R <= 256 = blockDim
    const int rr = threadIdx.x / R, j = threadIdx.x % R;
    if (rr >= rpp) return;
    for (int64_t k = (int64_t)blockIdx.x * rpp + rr; k < I; k += (int64_t)gridDim.x * rpp) {
        float *g = G + k * ld + j;
        *g = (float)((double)*g + c[j]);
    }
}

template <typename FT>
spt_status launch_colsums(const void *const *factors, const int64_t *dims, int d, int ld, int R, double *cs,
                          cudaStream_t st) {
    for (int l = 0; l < d; ++l) {
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(dims[l], (int64_t)sm_count() * 4));
        colsum_kernel<FT><<<blocks, 256, 0, st>>>((const FT *)factors[l], dims[l], ld, R, cs + (size_t)l * R);
        SPT_LAUNCH_CHECK("colsum_kernel");
    }
    return SPT_OK;
}

}  // namespace
}  // namespace spt

using namespace spt;

extern "C" {

spt_status gcp_gradient(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank, int ld,
                        int loss, float *grad, double *loss_out, void *stream) {
    if (!t || !factors || !grad) return fail(SPT_EINVAL, "gcp_gradient: NULL argument");
    if (mode < 0 || mode >= t->d) return fail(SPT_EINVAL, "gcp_gradient: mode out of range");
    if (t->d < 2 || t->d > SPT_MAX_KERNEL_ORDER) return fail(SPT_EUNSUPPORTED, "gcp_gradient: order must be 2..5");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16)
        return fail(SPT_EUNSUPPORTED, "gcp_gradient: factors must be fp32, bf16 or f16");
    if (loss < SPT_LOSS_POISSON || loss > SPT_LOSS_GAUSSIAN) return fail(SPT_EINVAL, "gcp_gradient: unknown loss");
    if (rank < 1 || rank > 256) return fail(SPT_EUNSUPPORTED, "gcp_gradient: rank must be in [1, 256]");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "gcp_gradient: ld must be >= rank and a multiple of 8");
    if (((uintptr_t)grad & 15) || ((uintptr_t)loss_out & 7))
        return fail(SPT_EINVAL, "gcp_gradient: grad not 16-byte or loss_out not 8-byte aligned");
    for (int m = 0; m < t->d; ++m)
        if (!factors[m] || ((uintptr_t)factors[m] & 15))
            return fail(SPT_EINVAL, "gcp_gradient: a factor pointer is NULL or not 16-byte aligned");
    if (!t->sorted_buf[mode])
        return fail(SPT_ESTATE, "gcp_gradient: needs the mode-sorted copy (build_mode_permutation)");
    spt_schedule s = default_schedule(t, mode, fdt, rank);
    s.scatter = SPT_SCATTER_SORTED;
    s.warps_per_cta = std::min(s.warps_per_cta, 8);  // gcp_kernel's launch bound: 256 threads
    if (s.lanes_per_nnz * s.chunks * 4 < rank) {  // the default rule covers R <= 256 in one block
        s.lanes_per_nnz = 32;
        s.chunks = 2;
    }
    spt_status c = check_schedule(t, mode, fdt, rank, s);
    if (c) return c;
    cudaStream_t st = (cudaStream_t)stream;
    if (loss_out) SPT_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(double), st));
    GcpArgs g{factors[mode], loss, loss_out};
    c = launch_mttkrp(t, mode, factors, fdt, rank, ld, nullptr, grad, s, st, &g);
    if (c) return c;
    if (loss != SPT_LOSS_POISSON) return SPT_OK;
    double *cs = nullptr;
    c = dmalloc((void **)&cs, sizeof(double) * (size_t)t->d * rank, st);
    if (c) return c;
    cudaError_t e = cudaMemsetAsync(cs, 0, sizeof(double) * (size_t)t->d * rank, st);
    if (e == cudaSuccess) {
        c = fdt == SPT_F32    ? launch_colsums<float>(factors, t->dims, t->d, ld, rank, cs, st)
            : fdt == SPT_BF16 ? launch_colsums<__nv_bfloat16>(factors, t->dims, t->d, ld, rank, cs, st)
                              : launch_colsums<__half>(factors, t->dims, t->d, ld, rank, cs, st);
        if (!c) {
            const int64_t In = t->dims[mode];
            const int rpp = 256 / rank;
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((In + rpp - 1) / rpp, sm_count() * 8));
            poisson_dense_kernel<<<blocks, 256, 0, st>>>(grad, In, ld, rank, cs, t->d, mode, loss_out);
            e = cudaGetLastError();
        }
    }
    dfree(cs, st);
    if (c) return c;
    if (e != cudaSuccess) return cuda_fail(e, "gcp_gradient");
    return SPT_OK;
}

}  // extern "C"

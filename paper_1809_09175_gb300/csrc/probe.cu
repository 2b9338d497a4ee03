// probe.cu -- STREAM-style copy (the bandwidth denominator the paper takes
// from STREAM, Sec. 7), an FMA-rate probe (the arithmetic denominator of the
// fp64 path, which is bound by GB300's fp64 units rather than by memory) and
// fp32 -> 16-bit factor storage conversion.
#include "internal.h"

namespace spt {
namespace {

// Persistent grid-stride copy, four independent 16-byte loads in flight per
// thread before the stores.
__global__ void __launch_bounds__(512) stream_copy_kernel(const uint4 *__restrict__ src,
                                                          uint4 *__restrict__ dst, int64_t n16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        uint4 a = __ldcs(src + i);
        uint4 b = __ldcs(src + i + stride);
        uint4 c = __ldcs(src + i + 2 * stride);
        uint4 d = __ldcs(src + i + 3 * stride);
        __stcs(dst + i, a);
        __stcs(dst + i + stride, b);
        __stcs(dst + i + 2 * stride, c);
        __stcs(dst + i + 3 * stride, d);
    }
    for (; i < n16; i += stride) __stcs(dst + i, __ldcs(src + i));
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Eight independent FMA chains per thread, `iters` steps each; the chains
// converge to c / (1 - b) and their sum is stored only if it equals an
// impossible value, which keeps them live.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T b, T c, double *sink) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x & 7) + (T)k;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma_t(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (T)-1) *sink = (double)s;
}

__global__ void convert_bf16_kernel(const float *src, __nv_bfloat16 *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void convert_f16_kernel(const float *src, __half *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

__global__ void convert_f32_kernel(const float *src, float *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
}  // namespace
}  // namespace spt

using namespace spt;

extern "C" {

spt_status spt_stream_copy(const void *src, void *dst, size_t bytes, void *stream) {
    if (!src || !dst) return fail(SPT_EINVAL, "spt_stream_copy: NULL pointer");
    if ((bytes & 15) || ((uintptr_t)src & 15) || ((uintptr_t)dst & 15))
        return fail(SPT_EINVAL, "spt_stream_copy: pointers and size must be 16-byte multiples");
    if (!bytes) return SPT_OK;
    const int64_t n16 = (int64_t)(bytes / 16);
    const int blocks = sm_count() * 4;
    stream_copy_kernel<<<blocks, 512, 0, (cudaStream_t)stream>>>((const uint4 *)src, (uint4 *)dst, n16);
    SPT_LAUNCH_CHECK("stream_copy_kernel");
    return SPT_OK;
}

spt_status spt_fma_probe(spt_dtype dt, int64_t iters, double *sink, double *flops, void *stream) {
    if (!sink || !flops || iters < 1) return fail(SPT_EINVAL, "spt_fma_probe: bad argument");
    if (dt != SPT_F32 && dt != SPT_F64) return fail(SPT_EINVAL, "spt_fma_probe: dtype must be SPT_F32 or SPT_F64");
    const int blocks = sm_count() * 8, threads = 256;
    cudaStream_t st = (cudaStream_t)stream;
    if (dt == SPT_F64)
        fma_probe_kernel<double><<<blocks, threads, 0, st>>>(iters, 0.999, 0.001, sink);
    else
        fma_probe_kernel<float><<<blocks, threads, 0, st>>>(iters, 0.999f, 0.001f, sink);
    SPT_LAUNCH_CHECK("fma_probe_kernel");
    *flops = 2.0 * 8.0 * (double)iters * (double)blocks * threads;
    return SPT_OK;
}

spt_status spt_convert_f32(const float *src, void *dst, spt_dtype fdt, int64_t n, void *stream) {
    if ((!src || !dst) && n > 0) return fail(SPT_EINVAL, "spt_convert_f32: NULL pointer");
    if (n <= 0) return SPT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8));
    switch (fdt) {
    case SPT_BF16: convert_bf16_kernel<<<blocks, 256, 0, st>>>(src, (__nv_bfloat16 *)dst, n); break;
    case SPT_F16: convert_f16_kernel<<<blocks, 256, 0, st>>>(src, (__half *)dst, n); break;
    case SPT_F32: convert_f32_kernel<<<blocks, 256, 0, st>>>(src, (float *)dst, n); break;
    default: return fail(SPT_EINVAL, "spt_convert_f32: bad dtype");
    }
    SPT_LAUNCH_CHECK("convert kernel");
    return SPT_OK;
}

}  // extern "C"

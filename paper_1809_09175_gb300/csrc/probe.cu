// probe.cu -- STREAM-style copy (the bandwidth denominator the paper takes
// from STREAM, Sec. 6) and fp32 -> 16-bit factor storage conversion.
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

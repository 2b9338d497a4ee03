// probe_gather.cu -- factor-row gather probe: how fast can 64-byte factor
// rows (16 fp32 columns) be brought to the SMs for a stream of row indices,
// by three routes?  (Sec. 7 measures its kernels against STREAM; this probe
// measures the ceiling of the MTTKRP's gather step, the part the permuted
// traversal cannot stream.)
//   0  16-byte ld.global per lane, 4 lanes per row, 8 rows per warp
//      instruction (the MTTKRP kernel's gathers);
//   1  TMA cp.async.bulk.tensor tile::gather4 (four rows per instruction,
//      2-D tensor map) into double-buffered shared memory, read back with
//      16-byte shared loads;
//   2  one 1-D cp.async.bulk per row into the same buffers;
//   3  as 0, but the 8 groups of a warp instruction take 8 consecutive
//      nonzeros (rows repeated among neighbours then share a load).
// Each nonzero gathers one row of F1 (index r1[i]) and one of F2 (r2[i]) and
// multiplies them, as the 3-way MTTKRP does; the products are kept live by a
// store that never happens.
#include <cuda.h>

#include "internal.h"

namespace spt {
namespace {

constexpr int GP_NPW = 64;  // nonzeros per warp chunk
constexpr int GP_WPC = 4;   // warps per CTA

__device__ __forceinline__ void keep_live(const float4 &acc, float *sink) {
    if (acc.x == 12345.f) *sink = acc.y + acc.z + acc.w;
}

__device__ __forceinline__ void fma4(float4 &acc, const float4 &x, const float4 &y) {
    acc.x = fmaf(x.x, y.x, acc.x);
    acc.y = fmaf(x.y, y.y, acc.y);
    acc.z = fmaf(x.z, y.z, acc.z);
    acc.w = fmaf(x.w, y.w, acc.w);
}

// INTERLEAVED: the 8 groups of a warp instruction take 8 consecutive
// nonzeros (t * 8 + g) instead of 8 nonzeros a chunk's eighth apart
template <bool INTERLEAVED>
__global__ void __launch_bounds__(128) gather_ldg_kernel(const float *F1, const float *F2, const int32_t *r1,
                                                         const int32_t *r2, int64_t nchunk, float *sink) {
    const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
    const int64_t gw = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t ch = gw * nchunk / nw; ch < (gw + 1) * nchunk / nw; ++ch) {
#pragma unroll 4
        for (int t = 0; t < GP_NPW / 8; ++t) {
            const int64_t e = ch * GP_NPW + (INTERLEAVED ? t * 8 + g : g * (GP_NPW / 8) + t);
            const int a = __ldg(r1 + e), b = __ldg(r2 + e);
            fma4(acc, __ldg(reinterpret_cast<const float4 *>(F1 + (int64_t)a * 16) + l),
                 __ldg(reinterpret_cast<const float4 *>(F2 + (int64_t)b * 16) + l));
        }
    }
    keep_live(acc, sink);
}

// Shared memory of the staged kernels: 16 bytes of barriers per warp, then
// (128-byte aligned: a tensor copy's destination must be) per warp two
// stages of 2 x GP_NPW rows of 64 bytes.
constexpr size_t GP_STAGE_BYTES = 2 * GP_NPW * 64;
constexpr size_t GP_SMEM = 128 + 128 + (size_t)GP_WPC * 2 * GP_STAGE_BYTES;

template <int METHOD>
__global__ void __launch_bounds__(128) gather_staged_kernel(const __grid_constant__ CUtensorMap m1,
                                                            const __grid_constant__ CUtensorMap m2, const float *F1,
                                                            const float *F2, const int32_t *r1, const int32_t *r2,
                                                            int64_t nchunk, float *sink, int *status) {
    extern __shared__ __align__(128) unsigned char gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
    uint64_t *bars = reinterpret_cast<uint64_t *>(gsm) + 2 * warp;
    unsigned char *base = gsm + 128;
    base += (128u - (smem_u32(base) & 127u)) & 127u;
    float *rows = reinterpret_cast<float *>(base + (size_t)warp * 2 * GP_STAGE_BYTES);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int64_t gw = blockIdx.x * (int64_t)GP_WPC + warp, nw = (int64_t)gridDim.x * GP_WPC;
    const int64_t c0 = gw * nchunk / nw, c1 = (gw + 1) * nchunk / nw;
    auto issue = [&](int64_t ch, int s) {
        float *dst = rows + s * (GP_STAGE_BYTES / 4);
        if (lane == 0) mbar_arrive_expect_tx(&bars[s], (uint32_t)GP_STAGE_BYTES);
        __syncwarp();
        if (METHOD == 1) {
            for (int j = lane; j < GP_NPW / 4; j += 32) {
                const int64_t e = ch * GP_NPW + 4 * j;
                const int4 a = *reinterpret_cast<const int4 *>(r1 + e);
                const int4 b = *reinterpret_cast<const int4 *>(r2 + e);
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst + 4 * j * 16)),
                    "l"(&m1), "r"(0), "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(smem_u32(&bars[s]))
                    : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst + (GP_NPW + 4 * j) * 16)),
                    "l"(&m2), "r"(0), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w), "r"(smem_u32(&bars[s]))
                    : "memory");
            }
        } else {
            for (int j = lane; j < GP_NPW; j += 32) {
                const int64_t e = ch * GP_NPW + j;
                bulk_g2s(dst + j * 16, F1 + (int64_t)r1[e] * 16, 64, &bars[s]);
                bulk_g2s(dst + (GP_NPW + j) * 16, F2 + (int64_t)r2[e] * 16, 64, &bars[s]);
            }
        }
    };
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c0 < c1) issue(c0, 0);
    int k = 0;
    for (int64_t ch = c0; ch < c1; ++ch, ++k) {
        const int s = k & 1;
        if (ch + 1 < c1) issue(ch + 1, s ^ 1);
        if (!__all_sync(0xffffffffu, mbar_wait(&bars[s], (uint32_t)(k >> 1) & 1u))) {
            // let the copies in flight land, report, leave
            if (lane == 0) atomicExch(status, SPT_DEV_TIMEOUT);
            if (ch + 1 < c1) mbar_wait(&bars[s ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            mbar_wait(&bars[s], (uint32_t)(k >> 1) & 1u);
            return;
        }
        const float *src = rows + s * (GP_STAGE_BYTES / 4);
#pragma unroll 4
        for (int t = 0; t < GP_NPW / 8; ++t) {
            const int e = g * (GP_NPW / 8) + t;
            fma4(acc, *reinterpret_cast<const float4 *>(src + e * 16 + 4 * l),
                 *reinterpret_cast<const float4 *>(src + (GP_NPW + e) * 16 + 4 * l));
        }
        __syncwarp();
        fence_proxy_async_smem();  // the stage is refilled by the copies issued next
    }
    keep_live(acc, sink);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// A 2-D tensor map over I rows of 16 fp32 columns, one-row boxes (the form
// tile::gather4 needs).
spt_status row_map(const float *F, int64_t I, CUtensorMap *map) {
    static EncodeTiledFn enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        SPT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn)
            return fail(SPT_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
        enc = reinterpret_cast<EncodeTiledFn>(fn);
    }
    const cuuint64_t dims[2] = {16, (cuuint64_t)I};
    const cuuint64_t strides[1] = {64};
    const cuuint32_t box[2] = {16, 1};
    const cuuint32_t es[2] = {1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(F), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(SPT_EINVAL, "spt_row_gather_probe: tensor map encoding failed");
    return SPT_OK;
}

}  // namespace
}  // namespace spt

using namespace spt;

extern "C" spt_status spt_row_gather_probe(int method, const float *F1, int64_t I1, const float *F2, int64_t I2,
                                           const int32_t *r1, const int32_t *r2, int64_t n, float *sink,
                                           int *status, void *stream) {
    if (method < 0 || method > 3) return fail(SPT_EINVAL, "spt_row_gather_probe: method must be 0..3");
    if (!F1 || !F2 || !r1 || !r2 || !sink || !status) return fail(SPT_EINVAL, "spt_row_gather_probe: NULL argument");
    if (I1 < 1 || I2 < 1 || I1 > INT32_MAX || I2 > INT32_MAX) return fail(SPT_EINVAL, "spt_row_gather_probe: bad row count");
    if (n < 0 || n % GP_NPW) return fail(SPT_EINVAL, "spt_row_gather_probe: n must be a multiple of 64");
    if (((uintptr_t)F1 | (uintptr_t)F2 | (uintptr_t)r1 | (uintptr_t)r2) & 15)
        return fail(SPT_EINVAL, "spt_row_gather_probe: pointers must be 16-byte aligned");
    if (n == 0) return SPT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nchunk = n / GP_NPW;
    int bps = 0;
    if (method == 0 || method == 3) {
        auto kf = method == 0 ? gather_ldg_kernel<false> : gather_ldg_kernel<true>;
        SPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kf, 32 * GP_WPC, 0));
        kf<<<std::max(1, bps) * sm_count(), 32 * GP_WPC, 0, st>>>(F1, F2, r1, r2, nchunk, sink);
        SPT_LAUNCH_CHECK("gather_ldg_kernel");
        return SPT_OK;
    }
    CUtensorMap m1, m2;
    memset(&m1, 0, sizeof(m1));
    memset(&m2, 0, sizeof(m2));
    if (method == 1) {
        spt_status s = row_map(F1, I1, &m1);
        if (!s) s = row_map(F2, I2, &m2);
        if (s) return s;
    }
    auto fn = method == 1 ? gather_staged_kernel<1> : gather_staged_kernel<2>;
    SPT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GP_SMEM));
    SPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 32 * GP_WPC, GP_SMEM));
    fn<<<std::max(1, bps) * sm_count(), 32 * GP_WPC, GP_SMEM, st>>>(m1, m2, F1, F2, r1, r2, nchunk, sink, status);
    SPT_LAUNCH_CHECK("gather_staged_kernel");
    return SPT_OK;
}

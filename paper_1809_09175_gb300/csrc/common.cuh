// common.cuh -- internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/spt.h"

#define SPT_MAX_ORDER 8
#define SPT_MAX_KERNEL_ORDER 5

// Device-side error codes written to a status word (never a trap).
#define SPT_DEV_OK 0
#define SPT_DEV_TIMEOUT 1
#define SPT_DEV_SINGULAR 2

// Iteration limit of every bounded spin-wait: each try_wait suspends for at
// most ~1 us (the hint below), so this bounds a wait to a few seconds.
#define SPT_WAIT_TRIES (1u << 22)
#define SPT_WAIT_HINT_NS 1000u

// Hot rows kept per mode for the atomic scatter's shared-memory copy.
#define SPT_HOT_MAX 256
#define SPT_HOT_MIN_COUNT 1024

struct ModeStats {
    bool valid = false;
    int64_t nonempty = 0;   // rows with at least one nonzero
    int64_t max_count = 0;  // nonzeros in the hottest row
    double sum_sq = 0.0;    // sum over rows of count^2
    int64_t runs_storage = 0; // row changes along storage order (+1)
};

struct spt_tensor_s {
    int device = 0;
    int d = 0;
    int64_t dims[SPT_MAX_ORDER] = {0};
    int64_t nnz = 0;
    bool coalesced = false;
    double xnorm2 = 0.0;
    // storage-order COO: one allocation, d index arrays then the values,
    // each segment 256-byte aligned.
    void *coo_buf = nullptr;
    int32_t *idx[SPT_MAX_ORDER] = {nullptr};
    float *vals = nullptr;
    // per mode: permutation and optional mode-sorted copy, stored as packed
    // records {row, other coordinates in increasing mode order, value bits}
    // of record_words(d) int32 words each
    int32_t *perm[SPT_MAX_ORDER] = {nullptr};
    void *sorted_buf[SPT_MAX_ORDER] = {nullptr};
    ModeStats stats[SPT_MAX_ORDER];
    // schedule chosen for a mode (by the autotuner or the selector) for one
    // (rank, dtype); used where the caller passes no schedule
    bool pref_set[SPT_MAX_ORDER] = {false};
    int pref_rank[SPT_MAX_ORDER] = {0};
    spt_dtype pref_fdt[SPT_MAX_ORDER] = {SPT_F32};
    spt_schedule pref[SPT_MAX_ORDER];
    int *dev_err = nullptr;  // device status word for kernels of this tensor
    // per mode: the hottest rows (most nonzeros, at least SPT_HOT_MIN_COUNT,
    // hottest first, ties in row order), up to SPT_HOT_MAX of them; the
    // atomic scatter adds their row sums into shared memory (see mttkrp_kernel)
    int32_t *hot_buf = nullptr;  // SPT_HOT_MAX entries per mode
    int nhot[SPT_MAX_ORDER] = {0};
    // nonzero counts of the listed rows and of the first row past the list
    // (hot_count[n][k], k <= nhot[n]; 0 past the candidates)
    int64_t hot_count[SPT_MAX_ORDER][SPT_HOT_MAX + 1] = {{0}};
    // sums over the mode's rows of count^2 and count^3 (the atomic scatter's
    // estimate of the rounding error of long fp32 chains of adds)
    double cnt_s2[SPT_MAX_ORDER] = {0.0};
    double cnt_s3[SPT_MAX_ORDER] = {0.0};
    // per mode, optional: the L2-blocked copy of the mode-sorted records --
    // grouped by blocks of blk_rows[n] rows of mode blk_mode[n] (each group in
    // the sorted copy's order, padded to a multiple of 4 records with
    // zero-valued copies of its last record), record offsets of the groups in
    // blk_off[n] (groups + 1 entries); the sorted traversal then runs one
    // launch per group, which gathers only that block of the mode's factor
    // optional: every nonzero in storage order as one record (its d
    // coordinates, the value's bits, zero padding to record_words(d) words),
    // read through perm_n by the perm_n traversal
    int32_t *srec = nullptr;
    void *blk_buf[SPT_MAX_ORDER] = {nullptr};
    int blk_mode[SPT_MAX_ORDER] = {-1, -1, -1, -1, -1, -1, -1, -1};
    int64_t blk_rows[SPT_MAX_ORDER] = {0};
    std::vector<int64_t> blk_off[SPT_MAX_ORDER];
};

// ---- host error handling -------------------------------------------------
namespace spt {
void set_error(const std::string &msg);
spt_status fail(spt_status st, const std::string &msg);
spt_status cuda_fail(cudaError_t e, const char *what);
int sm_count();
size_t seg_bytes(int64_t n, size_t elem);  // n*elem rounded up to 256
}  // namespace spt

#define SPT_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return spt::cuda_fail(e_, #call);    \
    } while (0)

#define SPT_LAUNCH_CHECK(what)                                      \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return spt::cuda_fail(e_, what);     \
    } while (0)

// ---- device helpers --------------------------------------------------------
namespace spt {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// 1-D bulk copy global -> shared (this CTA), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- thread-block clusters (distributed shared memory) ----
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of every CTA of the cluster; release/acquire
// orders the shared-memory writes before it against the reads after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// Shared-memory address `addr` of this CTA mapped to the same offset in the
// shared memory of cluster CTA `rank`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Atomic add into this CTA's shared memory.
__device__ __forceinline__ void red_add_shared(uint32_t addr, float v) {
    asm volatile("red.shared::cta.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(uint32_t addr, double v) {
    asm volatile("red.shared::cta.add.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// Atomic add into (possibly another CTA's) shared memory of the cluster.
__device__ __forceinline__ void red_add_cluster(uint32_t addr, float v) {
    asm volatile("red.relaxed.cluster.shared::cluster.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_cluster(uint32_t addr, double v) {
    asm volatile("red.relaxed.cluster.shared::cluster.add.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// Bounded wait for phase `parity` of `bar`: at most `tries` try_wait calls.
// Returns true when the phase completed, false when the budget ran out
// (tries = 0 gives up at once without looking).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t tries = SPT_WAIT_TRIES) {
    uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < tries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity), "r"(SPT_WAIT_HINT_NS)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Element traits: every lane works on chunks of VEC = 4 consecutive factor
// columns, loaded as one vector (16 bytes for fp32, 8 bytes for 16-bit
// types, two 16-byte loads for fp64) and widened to the accumulator type Acc
// (float, or double for fp64 factors).
template <typename T> struct Elem;
template <> struct Elem<float> {
    static constexpr int VEC = 4;
    static constexpr int BYTES = 4;
    typedef float Acc;
    typedef uint4 Raw;
    __device__ __forceinline__ static Raw load(const void *p) {
        return __ldg(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ static void widen(const Raw &r, float *o) {
        o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
        o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
    }
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr int VEC = 4;
    static constexpr int BYTES = 2;
    typedef float Acc;
    typedef uint2 Raw;
    __device__ __forceinline__ static Raw load(const void *p) {
        return __ldg(reinterpret_cast<const uint2 *>(p));
    }
    __device__ __forceinline__ static void widen(const Raw &r, float *o) {
        o[0] = bf16_lo(r.x); o[1] = bf16_hi(r.x); o[2] = bf16_lo(r.y); o[3] = bf16_hi(r.y);
    }
};
template <> struct Elem<__half> {
    static constexpr int VEC = 4;
    static constexpr int BYTES = 2;
    typedef float Acc;
    typedef uint2 Raw;
    __device__ __forceinline__ static Raw load(const void *p) {
        return __ldg(reinterpret_cast<const uint2 *>(p));
    }
    __device__ __forceinline__ static void widen(const Raw &r, float *o) {
        const uint32_t w[2] = {r.x, r.y};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[q]);
            float2 f = __half22float2(h);
            o[2 * q] = f.x;
            o[2 * q + 1] = f.y;
        }
    }
};

struct Raw64 {
    uint4 lo, hi;
};
template <> struct Elem<double> {
    static constexpr int VEC = 4;
    static constexpr int BYTES = 8;
    typedef double Acc;
    typedef Raw64 Raw;
    __device__ __forceinline__ static Raw load(const void *p) {
        Raw r;
        r.lo = __ldg(reinterpret_cast<const uint4 *>(p));
        r.hi = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
        return r;
    }
    __device__ __forceinline__ static void widen(const Raw &r, double *o) {
        o[0] = __hiloint2double((int)r.lo.y, (int)r.lo.x);
        o[1] = __hiloint2double((int)r.lo.w, (int)r.lo.z);
        o[2] = __hiloint2double((int)r.hi.y, (int)r.hi.x);
        o[3] = __hiloint2double((int)r.hi.w, (int)r.hi.z);
    }
};

}  // namespace spt

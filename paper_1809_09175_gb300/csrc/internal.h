// internal.h -- host-side functions shared between translation units.
#pragma once
#include <algorithm>
#include <string>

#include "common.cuh"

namespace spt {

spt_status dmalloc(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);
spt_status scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev,
                          cudaStream_t st);
spt_status radix_sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, int64_t n, int bits,
                            uint32_t *keys_out, int32_t *vals_out, cudaStream_t st);
spt_status coalesce_tensor(spt_tensor t, cudaStream_t st);
spt_status build_perm_mode(spt_tensor t, int n, bool index_only, cudaStream_t st);
spt_status compute_norm2(spt_tensor t, cudaStream_t st);

// MTTKRP launch with an explicit (validated) schedule; out is zeroed here.
spt_status launch_mttkrp(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                         int rank, int ld, const float *lambda, float *out,
                         const spt_schedule &sched, cudaStream_t st);
spt_status check_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank,
                          const spt_schedule &s);
spt_schedule default_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank);
int elem_bytes(spt_dtype fdt);
// forget the CUDA graphs captured for a tensor (its buffers changed or it died)
void drop_graphs(spt_tensor t);

}  // namespace spt

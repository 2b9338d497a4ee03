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
spt_status build_perm_mode(spt_tensor t, int n, bool index_only, cudaStream_t st, bool slice_order = false);
// t->srec: every nonzero in storage order as one packed record.
spt_status build_storage_records(spt_tensor t, cudaStream_t st);
// The L2-blocked copy of mode n's sorted records (t->blk_*[n]), blocks of
// block_rows rows of mode bm; needs the mode-sorted copy; synchronises `st`.
spt_status build_l2_blocks(spt_tensor t, int n, int bm, int64_t block_rows, cudaStream_t st);
spt_status compute_norm2(spt_tensor t, cudaStream_t st);
// The hot-row list of every mode (t->hot_buf, t->nhot); synchronises `st`.
spt_status build_hot_rows(spt_tensor t, cudaStream_t st);

// Generalised CP arguments of a gradient launch (see gcp_gradient).
struct GcpArgs {
    const void *fac_n;  // A^(n)
    int loss;
    double *loss_out;   // nullable
};

// MTTKRP launch with an explicit (validated) schedule; out is zeroed here.
// With gcp != NULL the launch runs the generalised CP gradient kernel
// instead (sorted traversal, one rank block).  det: deterministic sums (sorted
// traversal, one rank block): the rows a warp shares with its neighbours go
// to per-warp slots that a second kernel adds in slot order.
spt_status launch_mttkrp(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                         int rank, int ld, const void *lambda, void *out,
                         const spt_schedule &sched, cudaStream_t st, const GcpArgs *gcp = nullptr,
                         bool det = false);
spt_status check_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank,
                          const spt_schedule &s);
spt_schedule default_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank);
int elem_bytes(spt_dtype fdt);
// Bytes of the MTTKRP accumulator and output element (8 for fp64 factors, else 4).
int acc_bytes(spt_dtype fdt);
// Per-warp dynamic shared memory of a schedule (barriers, carry, staging).
size_t schedule_warp_smem(spt_tensor t, const spt_schedule &s, spt_dtype fdt);
// log2 of the smallest cluster (1, 2, 4 or 8 CTAs) whose shared memory holds
// the private output copy (ab-byte elements) of a mode of length In next to
// warp_smem bytes; -1 if none does.
int private_cluster_log2(int64_t In, int rank, size_t warp_smem, int ab);
// Candidate schedule q of the tuner's list for rank R, and whether it can run
// on (tensor, mode) with factors of type fdt.
spt_schedule candidate(int q, int rank);
bool candidate_valid(spt_tensor t, int mode, int rank, spt_dtype fdt, const spt_schedule &s, int q);
// Try budget of the kernels' staging waits for launches made from now on
// (spt_set_wait_tries; SPT_WAIT_TRIES by default).
uint32_t wait_tries();
// forget the CUDA graphs captured for a tensor (its buffers changed or it died)
void drop_graphs(spt_tensor t);

}  // namespace spt

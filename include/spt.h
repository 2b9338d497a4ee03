/*
 * spt.h -- C ABI of the GB300 sparse-tensor MTTKRP / CP-ALS library.
 *
 * Method: Phipps & Kolda, "Software for Sparse Tensor Decomposition on
 * Emerging Computing Architectures" (arXiv 1809.09175).  The tensor is a COO
 * list of P nonzeros x_i with coordinates (l_i1..l_id) (Sec. 3); the kernel
 * is the mode-n MTTKRP of Sec. 3 eq. (mttkrp); the permuted traversal is
 * Sec. 6 (Fig. "MTTKRP-C"); CP-ALS is the alternating least squares of Sec. 3.
 *
 * Conventions for every call
 *  - Nothing throws across the ABI.  Every call returns an spt_status; on
 *    failure spt_last_error() gives a message (per host thread).
 *  - "device" pointers are CUDA global memory of the current device (for
 *    example a torch tensor's data_ptr()); "host" pointers are CPU memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and do not synchronise the device, except where a call
 *    says it does.
 *  - Coordinates are 0-based int32; P < 2^31; order d in [1, 8] for storage,
 *    d in [1, 5] for the MTTKRP kernels.
 *  - Factor matrices are row-major I_m x ld with ld >= rank, ld a multiple
 *    of 8 elements (ld <= 2^28), base pointer 16-byte aligned.  Element type
 *    spt_dtype.
 *  - Asynchronous CUDA errors surface as SPT_ECUDA at a later call.
 */
#ifndef SPT_H
#define SPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spt_tensor_s *spt_tensor; /* opaque, library-owned */

typedef enum {
    SPT_OK = 0,
    SPT_EINVAL = 1,       /* bad argument (null pointer, order, mode, rank, ld, dtype, flags) */
    SPT_ERANGE = 2,       /* a coordinate outside [0, I_m) */
    SPT_ENOMEM = 3,       /* device or host allocation failed */
    SPT_ECUDA = 4,        /* a CUDA runtime call or kernel failed */
    SPT_EUNSUPPORTED = 5, /* valid request outside what the library implements */
    SPT_ESINGULAR = 6,    /* normal-equation matrix not positive definite (after ridge retry) */
    SPT_ETIMEOUT = 7,     /* a bounded device-side wait ran out */
    SPT_ESTATE = 8        /* the call needs an earlier step (e.g. a coalesced tensor) */
} spt_status;

/* Factor storage types.  SPT_F64 (fp64 factors, fp64 accumulation and
 * output: the precision of the paper's measurements, Sec. 7) is supported by
 * mttkrp and the schedule tools, not by cp_als_step or the batch. */
typedef enum { SPT_F32 = 0, SPT_BF16 = 1, SPT_F16 = 2, SPT_F64 = 3 } spt_dtype;

/* tensor_create_coo flags */
#define SPT_DEVICE_PTRS 1 /* idx / vals are device pointers (copied, not adopted) */
#define SPT_COALESCE 2    /* sum duplicate coordinates; output in lexicographic order */

/* build_mode_permutation flags */
#define SPT_PERM_INDEX_ONLY 1  /* keep only the permutation, not the mode-sorted copy */
#define SPT_PERM_SLICE_ORDER 2 /* order each slice of the mode-sorted copy by the next modes */

/* Scatter strategies of the MTTKRP (Sec. 4-6). */
typedef enum {
    SPT_SCATTER_AUTO = 0,   /* library choice (learned selector if loaded, else rule) */
    SPT_SCATTER_ATOMIC = 1, /* storage order, every row flush is an atomic add (Fig. MTTKRP-B) */
    SPT_SCATTER_PERM = 2,   /* permuted traversal through the mode-n permutation (Fig. MTTKRP-C) */
    SPT_SCATTER_SORTED = 3, /* permuted traversal over a mode-n-sorted copy of the nonzeros */
    SPT_SCATTER_PRIVATE = 4 /* storage order, row flushes added into a private copy of the
                             * output in shared memory (split over a cluster of up to 8
                             * CTAs when one CTA's cannot hold it), added to `out` at the
                             * end: the privatised scatter Sec. 8 proposes for short
                             * modes.  Needs no permutation; SPT_EINVAL when I_n rows
                             * of R floats do not fit 8 CTAs' shared memory. */
} spt_scatter;

/* A launch schedule of the MTTKRP kernel.
 *  lanes_per_nnz : 1,2,4,8,16,32 lanes share one nonzero (the paper's
 *                  vector_size, Tab. "sizes"); groups per warp = 32/lanes.
 *  chunks        : 1 or 2 four-column chunks per lane (one 16-byte load for
 *                  fp32, 8-byte for 16-bit factors); the rank block (the
 *                  paper's FBS) = lanes * chunks * 4 columns.
 *  nnz_per_group : nonzeros one lane group walks in order (the paper's
 *                  NZPTM); adjusted by the library for bank-conflict-free
 *                  staging.
 *  warps_per_cta : 1..16.
 *  ctas_per_sm   : persistent grid = SMs * ctas_per_sm; 0 = occupancy limit. */
typedef struct {
    int32_t scatter;
    int32_t lanes_per_nnz;
    int32_t chunks;
    int32_t nnz_per_group;
    int32_t warps_per_cta;
    int32_t ctas_per_sm;
} spt_schedule;

/* ---- errors ---------------------------------------------------------- */

/* Message of the last failed call on this host thread ("" if none). */
const char *spt_last_error(void);

/* ---- tensor ingest (Sec. 3, COO; Sec. 4.2 storage) --------------------- */

/* Create a COO tensor (Sec. 3: a P-vector of values and P x d coordinates).
 *  order     : d in [1, 8].
 *  dims      : host, d mode lengths I_m in [1, 2^31 - 1].
 *  nnz       : P in [0, 2^31 - 1].
 *  idx       : host array of d pointers; idx[m][i] = l_{i,m} (0-based int32),
 *              host memory, or device memory with SPT_DEVICE_PTRS.
 *  vals      : P float32 values x_i (host, or device with SPT_DEVICE_PTRS).
 *  flags     : SPT_DEVICE_PTRS | SPT_COALESCE.
 *  out       : receives the handle.
 * The tensor copies the data into library-owned device memory; the caller
 * keeps ownership of its buffers.  Coordinates are range-checked on the
 * device; this call synchronises `stream` to read the check and returns
 * SPT_ERANGE (creating nothing) if a coordinate is outside [0, I_m).
 * SPT_COALESCE sums duplicates (Sec. 3: an entry is the sum of the nonzeros
 * stored at its coordinate), leaving distinct coordinates in lexicographic
 * order; it is required by cp_als_step, whose fit needs ||X||. */
spt_status tensor_create_coo(int order, const int64_t *dims, int64_t nnz,
                             const int32_t *const *idx, const float *vals, int flags,
                             void *stream, spt_tensor *out);

/* Free a tensor and everything it owns (synchronises the device). */
spt_status tensor_destroy(spt_tensor t);

/* Shape of a tensor: order, dims (host, >= 8 entries), nnz (after
 * coalescing), and flags (bit SPT_COALESCE if coalesced). Any output may be NULL. */
spt_status tensor_info(spt_tensor t, int *order, int64_t *dims, int64_t *nnz, int *flags);

/* Copy the stored nonzeros out to caller device buffers: idx[m] (nnz int32
 * each, may be NULL to skip a mode) and vals (nnz float32, may be NULL). */
spt_status tensor_get_coo(spt_tensor t, int32_t *const *idx, float *vals, void *stream);

/* ||X||^2 in FP64 for a coalesced tensor (SPT_ESTATE otherwise). Host output. */
spt_status tensor_norm2(spt_tensor t, double *out);

/* Synchronise `stream` and read the tensor's device status word: SPT_OK, or
 * SPT_ETIMEOUT if a kernel's bounded wait ran out since the tensor was made
 * or since the last tensor_check that reported it (a reported status is
 * cleared, so later calls start clean). */
spt_status tensor_check(spt_tensor t, void *stream);

/* ---- mode permutations (Sec. 6) --------------------------------------- */

/* Build the mode-n permutation of Sec. 6: perm_n lists nonzero positions in
 * increasing mode-n coordinate, ties in storage order (a stable sort, done
 * by an on-device LSD radix sort).  mode = -1 builds all modes.  Unless
 * flags has SPT_PERM_INDEX_ONLY, the nonzeros are also copied in perm_n
 * order (a mode-sorted copy) so SPT_SCATTER_SORTED can stream them; with
 * SPT_PERM_SLICE_ORDER each slice's nonzeros in the copy are ordered by the
 * next modes (n+1, then n+2, cyclically; ties in storage order), so that
 * neighbouring nonzeros of a long slice repeat factor rows and share their
 * loads (two more radix sorts per mode).
 * Also records per-mode slice statistics used by the schedule selector.
 * Memory: 4P bytes per mode for perm_n, plus (4d + 4)P for the copy; the
 * radix sort borrows 16P bytes of temporary device memory. */
spt_status build_mode_permutation(spt_tensor t, int mode, int flags, void *stream);

/* keep = 1: pack the nonzeros, in storage order, into records of their d
 * coordinates and the value's bits (4 words each for d <= 3, 6 for d = 4, 5;
 * one array shared by every mode), so that the perm_n traversal
 * (SPT_SCATTER_PERM, the paper's Fig. MTTKRP-C) reads one record per nonzero
 * through perm_n instead of d + 1 separate scattered words; keep = 0 drops
 * them (the traversal then reads the coordinate arrays again).  Memory: 16P
 * or 24P bytes.  Stream-ordered.  Errors: SPT_EINVAL for a NULL tensor or a
 * keep other than 0 or 1. */
spt_status tensor_storage_records(spt_tensor t, int keep, void *stream);

/* Rows per block of build_mode_l2_blocks when block_rows < 0: 48 MB of
 * factor rows at 256 bytes a row (R = 64 in fp32), about a third of L2. */
#define SPT_L2_BLOCK_ROWS_DEFAULT 196608

/* Build the L2-blocked copy of mode `mode`'s sorted records: the records of
 * the mode-sorted copy grouped by blocks of `block_rows` consecutive rows of
 * mode `blocked_mode` (-1: the other mode with the most rows; block_rows < 0:
 * SPT_L2_BLOCK_ROWS_DEFAULT), each group keeping the copy's order (by mode
 * `mode`, then its slice order) and padded with zero-valued copies of its
 * last record to a multiple of 4 records.  While it exists, the sorted
 * traversal of that mode (mttkrp, its autotuning and CP-ALS; not the
 * deterministic, generalised-CP or batched calls, which keep the plain copy)
 * runs one launch per group, adding the rows it owns into the output, so the
 * gathers of the blocked mode's factor stay within one block at a time --
 * where that factor is much larger than L2, its rows are then read from DRAM
 * about once instead of once per nonzero.  block_rows == 0 drops the copy;
 * rebuilding the mode's permutation drops it too.  Needs the mode-sorted
 * copy (SPT_ESTATE otherwise).  Memory: the copy's size again plus 16 bytes
 * per group.  Synchronises `stream`.  Errors: SPT_EINVAL for a bad mode, a
 * blocked mode equal to `mode`, or more than 65536 blocks. */
spt_status build_mode_l2_blocks(spt_tensor t, int mode, int blocked_mode, int64_t block_rows, void *stream);

/* The L2-blocked copy of `mode`: blocked mode (-1 when there is none), rows
 * per block and number of groups.  Host outputs, each nullable. */
spt_status tensor_l2_blocks(spt_tensor t, int mode, int *blocked_mode, int64_t *block_rows, int64_t *groups);

/* A new tensor holding the nonzeros at positions [begin, end) of the mode-n
 * permutation of t (perm_n order: increasing mode-n coordinate), with t's
 * dims: the piece of t one process or GPU owns when the nonzeros are split
 * into contiguous ranges of perm_n (the multi-GPU distribution Sec. 8 names
 * as future work).  The shard is coalesced if t is (a subset of distinct
 * coordinates), with its own ||X||^2.  Needs build_mode_permutation(mode)
 * (SPT_ESTATE otherwise); SPT_EINVAL unless 0 <= begin <= end <= nnz.
 * Synchronises `stream`.  Free with tensor_destroy. */
spt_status tensor_create_shard(spt_tensor t, int mode, int64_t begin, int64_t end, void *stream,
                               spt_tensor *out);

/* Copy perm_n (P int32) to a caller device buffer. SPT_ESTATE if not built. */
spt_status tensor_get_permutation(spt_tensor t, int mode, int32_t *perm, void *stream);

/* Largest n mode_permutation_noalloc accepts (bounded by its 32 MiB static
 * scratch area: two key/position buffer pairs, the digit histogram and the
 * scan sums). */
#define SPT_NOALLOC_MAX_NNZ 1835008

/* The mode permutation of build_mode_permutation, computed without allocating
 * any device memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc/cudaFree at this point -- for
 * example code living inside a fixed device-memory budget owned by another
 * allocator, or code that must not incur the device-wide synchronisation of
 * cudaFree -- and therefore cannot let the library allocate sort buffers.
 *  keys   : device, n int32 mode coordinates (the tensor's l_{i,n}), each in
 *           [0, dim); other values give an unspecified (but in-bounds) order.
 *  n      : number of coordinates, 0 <= n <= SPT_NOALLOC_MAX_NNZ; larger n is
 *           rejected with SPT_EINVAL before any work is queued.
 *  dim    : the mode length I_n (sets the number of 8-bit radix passes).
 *  perm   : device, n int32 output: positions in increasing key order, equal
 *           keys in position order (the same result as perm_n).
 * The sort works in one static device array that is part of the library and
 * stays allocated on every GPU that has loaded it until the process exits.
 * Every call looks up that array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing); the first lookup on a
 * device also loads the library's device code there, so make the first call
 * on each device before any stream capture.
 * Every call uses the same array and leaves its last contents there; calls
 * that overlap on the GPU (other streams or host threads) race on it, so the
 * caller must order them.  Nothing is allocated or freed. */
spt_status mode_permutation_noalloc(const int32_t *keys, int64_t n, int64_t dim, int32_t *perm,
                                    void *stream);

/* ---- MTTKRP (Sec. 3 eq. mttkrp; Figs. MTTKRP-A/B/C) -------------------- */

/* Mode-n MTTKRP:  out(k, j) = lambda_j * sum_{i : l_in = k} x_i *
 *                             prod_{m != n} A^(m)(l_im, j)
 * for k < I_n, j < rank.
 *  factors : host array of d device pointers; factors[m] is A^(m), row-major
 *            I_m x ld of type fdt.  factors[mode] is not read (may be NULL).
 *  rank    : R >= 1.  ld : row stride of the factors and of out (elements,
 *            multiple of 8, >= rank).
 *  lambda  : device, rank weights (float32; float64 when fdt is SPT_F64), or
 *            NULL for all ones.
 *  out     : device I_n x ld, float32 (float64 when fdt is SPT_F64), 16-byte
 *            aligned; overwritten (columns >= rank set to 0).
 *  sched   : NULL = library choice; else the schedule to run (SPT_SCATTER_PERM
 *            and SPT_SCATTER_SORTED need build_mode_permutation(mode)).
 * Accumulation is float32 (float64 for SPT_F64).  The atomic and permuted
 * strategies add in different orders, so results agree to rounding, not bit
 * for bit. */
spt_status mttkrp(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank,
                  int ld, const void *lambda, void *out, const spt_schedule *sched,
                  void *stream);

/* Deterministic mode-n MTTKRP: arguments and result as mttkrp(), but the
 * sums are added in an order fixed by the tensor, the schedule and the GPU's
 * SM count, so repeated calls give bit-identical out.  The sorted traversal
 * with one rank block: rows inside a warp's range of nonzeros have one
 * writer; the two boundary rows of each range are written to per-warp slots
 * (scratch allocated and freed on `stream`) and a second kernel stores each
 * such row as the sum of its slots in warp order, in place of atomics.
 *  sched : NULL = the library's schedule made sorted (lanes widened to 32 if
 *          needed); else SPT_SCATTER_SORTED with lanes_per_nnz * chunks * 4
 *          >= rank (SPT_EINVAL otherwise).
 * SPT_ESTATE without the mode-sorted copy (build_mode_permutation);
 * SPT_EUNSUPPORTED for rank > 256. */
spt_status mttkrp_deterministic(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                                int rank, int ld, const void *lambda, void *out,
                                const spt_schedule *sched, void *stream);

/* Bytes of device workspace mttkrp_from_host needs for these modes (host
 * logic): the factors the listed modes read and one output per listed mode,
 * each 256-byte aligned. */
spt_status mttkrp_from_host_workspace_size(spt_tensor t, int nmodes, const int *modes, spt_dtype fdt,
                                           int rank, int ld, size_t *bytes);

/* MTTKRP from host memory: copies the factors to the device, runs mttkrp()
 * (the library's schedule) for modes[0], modes[1], ... in that order and
 * copies each result back.  The copies run on two library-owned streams
 * (created on first use per device, kept until exit) and are overlapped with
 * the kernels: the factors are uploaded in the order the modes first need
 * them (every factor but A^(modes[0]) first), each kernel waits only for
 * the factors it reads, and each result is downloaded as soon as its kernel
 * ends, while the next mode runs.  Stream-ordered: `stream` completes after
 * the last download; host buffers must stay valid until then.  A call that
 * fails after queuing copies still orders `stream` after them, so the
 * workspace and host buffers may be released once `stream` is done.  Pinned (page-
 * locked) host buffers give the overlap; pageable ones work, with copies
 * that block the calling thread.
 *  modes     : host, nmodes distinct modes (1 <= nmodes <= order).
 *  factors   : host array of d HOST pointers; factors[m] is A^(m), I_m x ld of
 *              type fdt, row-major; may be NULL when no listed mode reads it.
 *  lambda    : device weights as for mttkrp(), or NULL.
 *  out       : host array of nmodes HOST pointers; out[q] receives the
 *              I_{modes[q]} x ld result of mode modes[q] (float32; float64 for
 *              SPT_F64), columns >= rank zero.
 *  workspace : device, >= mttkrp_from_host_workspace_size() bytes, 256-byte
 *              aligned; the call's device copies of the factors and results.
 * Errors as for mttkrp(); SPT_EINVAL for a repeated or out-of-range mode, a
 * NULL needed pointer, or a short or misaligned workspace. */
spt_status mttkrp_from_host(spt_tensor t, int nmodes, const int *modes, const void *const *factors,
                            spt_dtype fdt, int rank, int ld, const void *lambda, void *const *out,
                            void *workspace, size_t workspace_bytes, void *stream);

/* Record the schedule to use for (mode, fdt, rank) wherever no schedule is
 * passed (mttkrp with sched == NULL, cp_als_step), e.g. one chosen by
 * mttkrp_autotune or mttkrp_select.  s == NULL clears it.  The schedule is
 * validated now (SPT_EINVAL / SPT_ESTATE as for mttkrp). */
spt_status tensor_set_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank, const spt_schedule *s);

/* The schedule mttkrp() runs for sched == NULL (host logic, no launch). */
spt_status mttkrp_default_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank,
                                   spt_schedule *out);

/* Tab. "sizes" (Sec. 5): the GPU vector_size and factor block size FBS the
 * paper uses for rank R. Host logic. */
spt_status mttkrp_paper_sizes(int rank, int *vector_size, int *fbs);

/* The paper's fixed rule (Tab. "sizes": vector_size and FBS as functions of R),
 * mapped onto this kernel's schedule for the given scatter strategy. */
spt_status mttkrp_paper_schedule(int rank, spt_dtype fdt, int scatter, spt_schedule *out);

/* ---- schedule search: candidates, autotuner, features, learned selector -- */
/* Not in the paper, whose schedule is the fixed rule of Tab. "sizes". */

#define SPT_NUM_CANDIDATES 48 /* fixed list of candidate schedules per (tensor, mode, rank) */
#define SPT_NUM_FEATURES 12   /* per-mode features of tensor_mode_features() */

/* The candidate schedules for rank R (host logic): candidate q combines a
 * scatter strategy (sorted / atomic / perm / private), a lane layout (ceil(R/4) lanes
 * rounded to a power of two with one chunk, or half as many lanes with two
 * chunks), about 96, 192 or 384 nonzeros per warp chunk, and 4 or 8 warps per
 * CTA.  out: SPT_NUM_CANDIDATES schedules; valid (nullable): 1 where the
 * candidate can run on this tensor (its permutation / copy is built, it fits
 * shared memory, a private copy of the output fits a cluster; judged for
 * 4-byte accumulators, i.e. any fdt but SPT_F64, which mttkrp_autotune and
 * mttkrp_select check for themselves). */
spt_status mttkrp_candidates(spt_tensor t, int mode, int rank, spt_schedule *out, int *valid);

/* Time one schedule: a warm-up launch, then the fastest of `reps` launches
 * (CUDA events).  Arguments as mttkrp(); synchronises `stream`. *ms in ms. */
spt_status mttkrp_time_schedule(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                                int rank, int ld, void *out, const spt_schedule *sched, int reps,
                                float *ms, void *stream);

/* Exhaustive autotuner: time every valid candidate (mttkrp_time_schedule)
 * and the library's own rule (mttkrp_default_schedule without a recorded
 * preference), and return the fastest in *best (and its time in *best_ms).
 * times (nullable, SPT_NUM_CANDIDATES floats, host) receives every
 * candidate's time, -1 for invalid ones: the training data of the learned
 * selector.
 * `out` is scratch output (I_mode x ld float32).  Synchronises `stream`. */
spt_status mttkrp_autotune(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank,
                           int ld, void *out, int reps, spt_schedule *best, float *best_ms,
                           float *times, void *stream);

/* Per-mode features (host output, SPT_NUM_FEATURES floats): order, log2 I_n,
 * log2 (P / I_n), min(log2 P, 24), log2 R, factor element bytes, log2 of the
 * hottest slice over the mean nonempty slice, coefficient of variation of the
 * slice sizes, hottest-slice share of P, nonempty-slice fraction, log2 of the
 * mean run length of equal mode-n coordinates in storage order, and log2 of
 * the other factors' bytes over the 129 MB L2.  Needs build_mode_permutation(mode). */
spt_status tensor_mode_features(spt_tensor t, int mode, int rank, spt_dtype fdt, float *feat);

/* Sizes of the selector network h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
 * y = W3 h2 + b3 with parameters packed W1 (H1 x F), b1, W2 (H2 x H1), b2,
 * W3 (K x H2), b3 (row-major, float32). */
int64_t mlp_param_count(int F, int H1, int H2, int K);
/* Floats of the `work` buffer mlp_forward / mlp_loss_grad need for B samples. */
int64_t mlp_workspace_floats(int B, int F, int H1, int H2, int K);

/* Forward pass for B samples (rows of X, B x F, device) into Y (B x K). */
spt_status mlp_forward(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                       float *Y, float *work, void *stream);

/* Masked mean-squared error L = sum M (Y - T)^2 / sum M and its gradient
 * with respect to every parameter (packed like params) by back-propagation;
 * *loss is a device float.  All pointers device. */
spt_status mlp_loss_grad(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                         const float *T, const float *M, float *grads, float *loss, float *work,
                         void *stream);

/* One Adam step (bias-corrected, step >= 1) on n parameters. */
spt_status mlp_adam(int64_t n, float *params, const float *grads, float *m, float *v, float lr,
                    float beta1, float beta2, float eps, int step, void *stream);

/* Fused one-CTA inference for a few samples (the selector's path). */
spt_status mlp_infer(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                     float *Y, void *stream);

/* A trained selector: F = SPT_NUM_FEATURES, K = SPT_NUM_CANDIDATES, params
 * on the device; mean / std (host, F floats, nullable) normalise features. */
typedef struct {
    int F, H1, H2, K;
    const float *params;
    const float *mean;
    const float *std;
    float anchor_margin; /* >= 0: the outputs are log(candidate time / time of the
                          * schedule mttkrp() runs for sched == NULL), and that
                          * schedule is kept unless the best valid prediction is
                          * below -anchor_margin; < 0: the outputs are relative
                          * log times and the smallest always wins */
} spt_selector;

/* Choose a schedule with a trained selector: features -> network (own
 * inference kernel) -> the valid candidate with the smallest predicted time,
 * or (anchor_margin >= 0) mttkrp_default_schedule's choice when no candidate
 * is predicted to beat it by more than the margin.  pred (nullable, host,
 * SPT_NUM_CANDIDATES) receives the predictions.  Synchronises `stream`. */
spt_status mttkrp_select(spt_tensor t, int mode, spt_dtype fdt, int rank, const spt_selector *sel,
                         spt_schedule *out, float *pred, void *stream);

/* ---- batched MTTKRP: many tensors, all modes, one persistent launch ----- */

typedef struct spt_batch_s *spt_batch; /* opaque, library-owned */

/* One tensor of a batch.  The MTTKRP definition is that of mttkrp() (unit
 * weights); the traversal is the permuted one over the mode-sorted copy
 * (Sec. 6), so every listed mode needs build_mode_permutation() without
 * SPT_PERM_INDEX_ONLY.
 *  tensor  : order 2..5.   mode : -1 = every mode, else one mode.
 *  rank, ld: as for mttkrp(); factors and outputs share ld.
 *  factors : host array of d device pointers (the batch's dtype), I_m x ld.
 *  outs    : host array of device float32 outputs I_n x ld: d entries for
 *            mode -1 (outs[n] for mode n), else one entry.
 *  scheds  : NULL for the library choice, else d entries (or one for a
 *            single mode); their scatter field is ignored. */
typedef struct {
    spt_tensor tensor;
    int mode;
    int rank;
    int ld;
    const void *const *factors;
    float *const *outs;
    const spt_schedule *scheds;
} spt_batch_item;

/* Build a batch: one task per (tensor, mode); tasks are grouped by kernel
 * class (chunks per lane, and order 5 apart from orders 2..4: one class for
 * tensors of order up to 4 and ranks up to 128 with the library's
 * schedules), and each class's task chunks, cut into blocks of 8, form its
 * work list.  Copies the task tables to the device
 * (synchronous); the pointers are captured, so the tensors, factors and
 * outputs must outlive the batch and keep their addresses. */
spt_status mttkrp_batch_create(int count, const spt_batch_item *items, spt_dtype fdt, spt_batch *out);

/* Run every task: one zero-fill kernel for the outputs and counters, then
 * one persistent kernel per class whose warps claim blocks of chunks from
 * the class's device counter and run each with the routine of its task's
 * order.  On a non-default stream the launches are
 * captured in a CUDA graph at the first call and replayed afterwards; on the
 * legacy default stream they are launched directly. */
spt_status mttkrp_batch_run(spt_batch b, void *stream);

/* Tasks, work items (chunks) and persistent CTAs (the largest class's grid)
 * of a batch.  Host outputs. */
spt_status mttkrp_batch_info(spt_batch b, int64_t *tasks, int64_t *items, int *blocks);

/* Synchronise `stream` and read the batch kernel's status word (SPT_ETIMEOUT
 * if a bounded wait ran out); a reported status is cleared. */
spt_status mttkrp_batch_check(spt_batch b, void *stream);

/* Free a batch (synchronises the device). */
spt_status mttkrp_batch_destroy(spt_batch b);

/* ---- generalised CP gradient (Sec. 8: count and binary data) ---------- */

/* Losses of gcp_gradient, with m the model value sum_j prod_l A^(l)(e_l, j)
 * of an entry e and x its value. */
typedef enum {
    SPT_LOSS_POISSON = 0,         /* f = m - x log m over EVERY entry of the tensor (x = 0 off the
                                   * stored coordinates; duplicates add); needs m > 0 at the
                                   * stored entries (e.g. nonnegative factors) */
    SPT_LOSS_BERNOULLI_LOGIT = 1, /* f = log(1 + e^m) - x m over the STORED entries only (store
                                   * sampled zeros explicitly; each stored copy is one term) */
    SPT_LOSS_GAUSSIAN = 2         /* f = (m - x)^2 over the stored entries */
} spt_loss;

/* Gradient of the generalised CP loss F = sum f(x_e, m_e) with respect to
 * A^(n):  grad(k, j) = sum_{e : e_n = k} df/dm(x_e, m_e) prod_{l != n} A^(l)(e_l, j)
 * -- an MTTKRP whose values are df/dm at the model value (computed with
 * A^(n) itself), run over the mode-sorted copy.  For SPT_LOSS_POISSON the
 * entries off the stored coordinates (df/dm = 1) contribute
 * prod_{l != n} colsum_l(j) to every row, added in fp64.
 *  factors : host array of d device pointers, ALL read (including factors[mode]),
 *            row-major I_m x ld, fdt in {SPT_F32, SPT_BF16, SPT_F16}.
 *  rank    : 1..256 (one rank block of the kernel).  ld as for mttkrp.
 *  grad    : device float32 I_n x ld, 16-byte aligned; overwritten (columns >= rank 0).
 *  loss_out: device double or NULL; set to F (fp32 terms, fp64 sums).
 * Needs build_mode_permutation(mode) (SPT_ESTATE otherwise); order 2..5.
 * Allocates a d x rank fp64 scratch (stream-ordered) for the Poisson loss. */
spt_status gcp_gradient(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank, int ld,
                        int loss, float *grad, double *loss_out, void *stream);

/* ---- CP-ALS (Sec. 3) -------------------------------------------------- */

/* Workspace bytes cp_als_step needs for this tensor, rank and ld. */
spt_status cp_als_workspace_size(spt_tensor t, int rank, int ld, size_t *bytes);

/* One CP-ALS iteration over all modes n = 0..d-1 in order (Sec. 3, ALS):
 *   V = MTTKRP_n(X, A) (unit weights); H = elementwise product over m != n of
 *   A^(m)T A^(m) (FP64); H^-1 in FP64 by symmetric elimination, whose pivots
 *   are the squared diagonal of the Cholesky factor H = L L^T (so it succeeds
 *   exactly when H is positive definite; one retry with a ridge of
 *   1e-12 trace(H)/R); A^(n) = V H^-1; lambda_j = ||A^(n)(:,j)||_2 (FP64) and
 *   A^(n)(:,j) /= lambda_j; 16-bit factors are rounded (nearest even) after
 *   normalising.  After the last mode, fit = 1 - ||X - M|| / ||X|| with
 *   ||M||^2 = lambda^T (*_m G_m) lambda and <X, M> = sum_{k,j} V(k,j) lambda_j
 *   A^(d)(k,j) from the last mode's V (FP64 reductions).
 *  factors   : host array of d device pointers, I_m x ld, type fdt; updated.
 *  lambda    : device, rank doubles (output).
 *  fit_out   : device double (output) or NULL.
 *  workspace : device, >= cp_als_workspace_size() bytes, 256-byte aligned.
 * Needs a coalesced tensor (SPT_ESTATE) and rank <= 128 (SPT_EUNSUPPORTED).
 * SPT_ESINGULAR is reported by the next call (or cp_als_status) because the
 * solve runs on the device; the factors of a singular mode are left as V. */
spt_status cp_als_step(spt_tensor t, void *const *factors, spt_dtype fdt, int rank, int ld,
                       double *lambda, double *fit_out, void *workspace, size_t workspace_bytes,
                       void *stream);

/* The steps of one CP-ALS mode update (Sec. 3 ALS; cp_als_step runs the same
 * kernels), one call each, for a caller that splits the nonzeros -- and so
 * the rows of V -- across processes or GPUs and exchanges the partial sums
 * itself (the multi-GPU distribution Sec. 8 names as future work): per mode
 * n, V = the mode-n MTTKRP of its nonzeros (mttkrp) summed over the pieces,
 * then cp_als_hinv, cp_als_apply on its rows of V, a sum of colsq over the
 * pieces, cp_als_normalize, cp_als_gram on its rows of the new factor, a sum
 * of the Grams over the pieces, and the factor rows gathered back; after
 * the last mode, cp_als_fit.  Stream-ordered, no synchronisation.
 *
 * cp_als_hinv: H = elementwise product over m != mode of the R x R FP64
 *   Grams G (device, order * R * R doubles, G_m at G + m R R); hinv (device,
 *   R * R float32) = H^-1 by Gauss-Jordan elimination in FP64 without
 *   pivoting, whose pivots are the squared diagonal of the Cholesky factor
 *   H = L L^T, with one retry at a ridge of 1e-12 trace(H)/R.  If a pivot is
 *   <= 0 after the ridge (H not positive definite), *status (device int) is
 *   set to 2 and hinv to the identity. */
spt_status cp_als_hinv(const double *G, int order, int mode, int rank, float *hinv, int *status, void *stream);

/* cp_als_apply: A32 = V hinv for `rows` rows of V (device, rows x ld float32,
 *   columns >= rank zero) into A32 (device, rows x ld float32, columns >=
 *   rank not written), and colsq[j] += sum over the rows of A32(:, j)^2
 *   (device, rank doubles; the caller zeroes it).  FP32 FMAs, FP64 sums. */
spt_status cp_als_apply(const float *V, int64_t rows, int ld, int rank, const float *hinv, float *A32,
                        double *colsq, void *stream);

/* cp_als_normalize: lambda_j = sqrt(colsq_j) (device, rank doubles, the
 *   sums over ALL rows), A = A32 / lambda in the factor type fdt (device,
 *   rows x ld, padding columns zero, 16-bit types rounded to nearest even; a
 *   zero column is kept).  With V and inner (both device, or both NULL):
 *   inner += sum V(k, j) lambda_j A(k, j) over these rows (the <X, M> term of
 *   the fit from the last mode's V; the caller zeroes it). */
spt_status cp_als_normalize(const float *A32, const float *V, int64_t rows, int ld, int rank, const double *colsq,
                            void *A, spt_dtype fdt, double *lambda, double *inner, void *stream);

/* cp_als_gram: G += A^T A over `rows` rows of A (device, rows x ld of fdt),
 *   G device R x R FP64 (FP32 partial sums over at most 256 rows, added in
 *   FP64; the caller zeroes G). */
spt_status cp_als_gram(const void *A, int64_t rows, int ld, int rank, spt_dtype fdt, double *G, void *stream);

/* cp_als_fit: fit = 1 - sqrt(max(0, xnorm2 + ||M||^2 - 2 inner)) / sqrt(xnorm2)
 *   with ||M||^2 = lambda^T (*_m G_m) lambda (G: order Grams as for
 *   cp_als_hinv); *inner (device double, the summed <X, M>) is read and then
 *   set to 0; *fit is a device double. */
spt_status cp_als_fit(const double *G, int order, int rank, const double *lambda, double *inner, double xnorm2,
                      double *fit, void *stream);

/* Device status word of the last cp_als_step on this workspace (synchronises
 * `stream`): SPT_OK or SPT_ESINGULAR. */
spt_status cp_als_status(void *workspace, void *stream);

/* ---- utilities -------------------------------------------------------- */

/* STREAM-style copy dst[0:bytes) = src[0:bytes) with this library's own
 * kernel (16-byte vector loads/stores, persistent grid); the bandwidth
 * denominator that Sec. 7 takes from STREAM. bytes % 16 == 0,
 * both pointers 16-byte aligned. */
spt_status spt_stream_copy(const void *src, void *dst, size_t bytes, void *stream);

/* FMA-rate probe (no counterpart in the paper): enqueue a kernel in which
 * every thread of a grid of 8 CTAs of 256 threads per SM runs 8 independent
 * FMA chains of `iters` steps in dt (SPT_F32 or SPT_F64).  *flops (host)
 * receives the floating-point operations it performs (2 per FMA); time the
 * launch with events on `stream` to get the device's FMA throughput.  sink is
 * a device double that the kernel never writes in practice. */
spt_status spt_fma_probe(spt_dtype dt, int64_t iters, double *sink, double *flops, void *stream);

/* Factor-row gather probe (no counterpart in the paper; the ceiling of the
 * MTTKRP's gather step): for i < n, bring row r1[i] of F1 and row r2[i] of
 * F2 (row-major, 16 float32 columns = 64 bytes per row, I1 and I2 rows) to
 * the SMs and multiply them, by
 *   method 0: 16-byte global loads, 4 lanes per row (the MTTKRP kernel's way);
 *   method 1: TMA tile::gather4 into shared memory (four rows per instruction);
 *   method 2: one 1-D bulk copy per row into shared memory;
 *   method 3: as 0, with the 8 groups of a warp instruction on 8 consecutive
 *             nonzeros (neighbours that repeat a row then share its load).
 * Enqueues one launch on `stream`; time it with events.  n a multiple of 64;
 * every pointer device, 16-byte aligned; sink a device float the kernel
 * never writes in practice; status a device int set to 1 if a bounded wait
 * of methods 1 and 2 ran out. */
spt_status spt_row_gather_probe(int method, const float *F1, int64_t I1, const float *F2, int64_t I2,
                                const int32_t *r1, const int32_t *r2, int64_t n, float *sink, int *status,
                                void *stream);

/* Convert n float32 values to fdt storage (round to nearest even). */
spt_status spt_convert_f32(const float *src, void *dst, spt_dtype fdt, int64_t n, void *stream);

/* Try budget of the bounded waits in the MTTKRP kernels (the staging
 * barriers of the bulk copies; failure detection, no counterpart in the
 * paper).  A wait that runs out of tries sets the tensor's (or batch's)
 * status word, lets the warp's copies in flight land (with the full default
 * budget), and ends the warp's work; tensor_check / mttkrp_batch_check then
 * report SPT_ETIMEOUT.  Applies to launches made after the call, library-wide
 * (captured CUDA graphs and batch tables keep the budget they were made with).
 *  tries : -1 restores the default (2^22 tries of about 1 us each); 0 makes
 *          every such wait give up at once, which is how the timeout path is
 *          tested without a fault; otherwise the number of try_wait calls.
 * SPT_EINVAL for tries < -1 or >= 2^32.  Host logic, no launch. */
spt_status spt_set_wait_tries(int64_t tries);

/* Number of SMs of the current device and this library's build arch (e.g. 103). */
spt_status spt_device_info(int *sm_count, int *arch);

#ifdef __cplusplus
}
#endif
#endif /* SPT_H */

// tune.cu -- schedule search for the MTTKRP: the candidate list, the
// exhaustive autotuner (which also produces the timing data the learned
// selector is trained on), per-mode features, and selection by a trained
// network.  None of this is in the paper, whose schedule is the fixed rule of
// Tab. "sizes" (Sec. 5); that rule is kept (mttkrp_paper_schedule) as the
// baseline the learned selector is measured against.
#include <cmath>
#include <vector>

#include "internal.h"
#include "mttkrp_kernel.cuh"

namespace spt {

// candidate q = ((scatter_i * 2 + lanes_i) * 3 + npw_i) * 2 + warps_i, scatter_i in 0..3
static const int kScatters[4] = {SPT_SCATTER_SORTED, SPT_SCATTER_ATOMIC, SPT_SCATTER_PERM,
                                 SPT_SCATTER_PRIVATE};
static const int kNpw[3] = {96, 192, 384};
static const int kWarps[2] = {4, 8};

spt_schedule candidate(int q, int rank) {
    spt_schedule s{};
    const int wi = q % 2, ni = (q / 2) % 3, li = (q / 6) % 2, si = q / 12;
    s.scatter = kScatters[si];
    const int need = (rank + 3) / 4;  // four-column chunks
    int L0 = 1;
    while (L0 < need && L0 < 32) L0 <<= 1;
    const int C0 = need > 32 ? 2 : 1;
    if (li == 0) {
        s.lanes_per_nnz = L0;
        s.chunks = C0;
    } else {  // half the lanes, two chunks each (same rank block, more groups)
        s.lanes_per_nnz = std::max(1, L0 / 2);
        s.chunks = 2;
    }
    const int G = 32 / s.lanes_per_nnz;
    s.nnz_per_group = std::max(4, kNpw[ni] / G);
    s.warps_per_cta = kWarps[wi];
    s.ctas_per_sm = 0;
    return s;
}

bool candidate_valid(spt_tensor t, int mode, int rank, spt_dtype fdt, const spt_schedule &s, int q) {
    const int li = (q / 6) % 2;
    const int need = (rank + 3) / 4;
    if (li == 1 && need <= 1) return false;  // nothing to halve
    if (s.scatter == SPT_SCATTER_SORTED && !t->sorted_buf[mode]) return false;
    if (s.scatter == SPT_SCATTER_PERM && !t->perm[mode]) return false;
    const size_t smem = schedule_warp_smem(t, s, fdt);
    if (smem > 227 * 1024) return false;
    if (s.scatter == SPT_SCATTER_PRIVATE && private_cluster_log2(t->dims[mode], rank, smem, acc_bytes(fdt)) < 0)
        return false;
    return true;
}

}  // namespace spt

using namespace spt;

extern "C" {

spt_status mttkrp_candidates(spt_tensor t, int mode, int rank, spt_schedule *out, int *valid) {
    if (!t || !out) return fail(SPT_EINVAL, "mttkrp_candidates: NULL argument");
    if (mode < 0 || mode >= t->d || rank < 1) return fail(SPT_EINVAL, "mttkrp_candidates: bad mode/rank");
    for (int q = 0; q < SPT_NUM_CANDIDATES; ++q) {
        out[q] = candidate(q, rank);
        if (valid) valid[q] = candidate_valid(t, mode, rank, SPT_F32, out[q], q) ? 1 : 0;
    }
    return SPT_OK;
}

spt_status mttkrp_time_schedule(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt,
                                int rank, int ld, void *out, const spt_schedule *sched, int reps,
                                float *ms, void *stream) {
    if (!t || !sched || !ms) return fail(SPT_EINVAL, "mttkrp_time_schedule: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SPT_CUDA(cudaEventCreate(&e0));
    SPT_CUDA(cudaEventCreate(&e1));
    spt_status s = mttkrp(t, mode, factors, fdt, rank, ld, nullptr, out, sched, stream);  // warm-up
    float best = INFINITY;
    for (int r = 0; r < std::max(1, reps) && s == SPT_OK; ++r) {
        cudaEventRecord(e0, st);
        s = mttkrp(t, mode, factors, fdt, rank, ld, nullptr, out, sched, stream);
        cudaEventRecord(e1, st);
        if (s) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { s = cuda_fail(e, "mttkrp_time_schedule"); break; }
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        best = std::min(best, x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    *ms = best;
    return SPT_OK;
}

spt_status mttkrp_autotune(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank,
                           int ld, void *out, int reps, spt_schedule *best, float *best_ms,
                           float *times, void *stream) {
    if (!t || !best) return fail(SPT_EINVAL, "mttkrp_autotune: NULL argument");
    if (mode < 0 || mode >= t->d || rank < 1) return fail(SPT_EINVAL, "mttkrp_autotune: bad mode/rank");
    float bms = INFINITY;
    int bq = -1;
    for (int q = 0; q < SPT_NUM_CANDIDATES; ++q) {
        const spt_schedule c = candidate(q, rank);
        float ms = -1.f;
        if (candidate_valid(t, mode, rank, fdt, c, q)) {
            spt_status s = mttkrp_time_schedule(t, mode, factors, fdt, rank, ld, out, &c, reps, &ms, stream);
            if (s) return s;
            if (ms < bms) { bms = ms; bq = q; }
        }
        if (times) times[q] = ms;
    }
    // the library's own rule is timed too, so the tuner never returns a
    // schedule slower than running without it (the rule's chunk sizes lie
    // between the candidates' and often win on large tensors)
    spt_schedule pick = bq >= 0 ? candidate(bq, rank) : spt_schedule{};
    const bool had_pref = t->pref_set[mode];
    t->pref_set[mode] = false;  // the rule itself, not a recorded choice
    const spt_schedule rule = default_schedule(t, mode, fdt, rank);
    t->pref_set[mode] = had_pref;
    if (check_schedule(t, mode, fdt, rank, rule) == SPT_OK) {
        float ms = -1.f;
        spt_status s = mttkrp_time_schedule(t, mode, factors, fdt, rank, ld, out, &rule, reps, &ms, stream);
        if (s) return s;
        if (ms < bms) {
            bms = ms;
            pick = rule;
            bq = SPT_NUM_CANDIDATES;
        }
    }
    if (bq < 0) return fail(SPT_EUNSUPPORTED, "mttkrp_autotune: no valid candidate");
    *best = pick;
    if (best_ms) *best_ms = bms;
    return SPT_OK;
}

spt_status tensor_mode_features(spt_tensor t, int mode, int rank, spt_dtype fdt, float *feat) {
    if (!t || !feat) return fail(SPT_EINVAL, "tensor_mode_features: NULL argument");
    if (mode < 0 || mode >= t->d || rank < 1) return fail(SPT_EINVAL, "tensor_mode_features: bad mode/rank");
    const ModeStats &ms = t->stats[mode];
    if (!ms.valid) return fail(SPT_ESTATE, "tensor_mode_features: build_mode_permutation(mode) first");
    const double P = std::max<double>(1.0, (double)t->nnz);
    const double In = (double)t->dims[mode];
    double other_rows = 0.0;
    for (int m = 0; m < t->d; ++m)
        if (m != mode) other_rows += (double)t->dims[m];
    const double eb = (double)elem_bytes(fdt);
    const double ne = std::max<double>(1.0, (double)ms.nonempty);
    const double mean_ne = P / ne;
    const double mean_all = P / In;
    const double var = std::max(0.0, ms.sum_sq / In - mean_all * mean_all);
    const double l2 = 129.0 * 1024 * 1024;
    feat[0] = (float)t->d;
    feat[1] = (float)std::log2(In);
    feat[2] = (float)std::log2(P / In);                   // mean slice length
    feat[3] = (float)std::min(24.0, std::log2(P));        // size, saturated: tails vanish beyond 16M
    feat[4] = (float)std::log2((double)rank);
    feat[5] = (float)eb;
    feat[6] = (float)std::log2(std::max(1.0, (double)ms.max_count / mean_ne));
    feat[7] = (float)(mean_all > 0 ? std::sqrt(var) / mean_all : 0.0);
    feat[8] = (float)((double)ms.max_count / P);
    feat[9] = (float)(ne / In);
    feat[10] = (float)std::log2(P / std::max<double>(1.0, (double)ms.runs_storage));
    feat[11] = (float)std::log2(std::max(1.0, other_rows * rank * eb) / l2);
    return SPT_OK;
}

}  // extern "C"

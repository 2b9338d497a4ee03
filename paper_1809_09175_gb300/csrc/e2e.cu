// e2e.cu -- MTTKRP from host memory: the factors go to the device, the
// listed modes' MTTKRPs run, the results come back, with the copies
// overlapped with the kernels.
//
// Three streams: the caller's stream runs the kernels; an upload stream
// copies the factors in the order the modes first need them, an event after
// each; a download stream copies each result back as soon as its kernel has
// finished.  For a 3-way tensor and modes 0, 1, 2 this hides the upload of
// A^(0) behind the mode-0 kernel and the download of V^(0) and V^(1) behind
// the next kernels; only the first d-1 uploads and the last download are
// exposed.
#include <mutex>

#include "internal.h"

namespace spt {
namespace {

constexpr size_t ALIGN = 256;

size_t round_up(size_t b) { return (b + ALIGN - 1) & ~(ALIGN - 1); }

// The upload and download streams of a device (created on first use and
// kept for the life of the process; calls from several host threads share
// them, which orders their copies but never their results: every
// dependency goes through the call's own events).
struct CopyStreams {
    cudaStream_t up = nullptr, down = nullptr;
};
std::mutex g_copy_mu;
CopyStreams g_copy[64];

spt_status copy_streams(CopyStreams *&cs) {
    int dev = 0;
    SPT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SPT_EUNSUPPORTED, "mttkrp_from_host: device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_copy_mu);
    CopyStreams &c = g_copy[dev];
    if (!c.up) SPT_CUDA(cudaStreamCreateWithFlags(&c.up, cudaStreamNonBlocking));
    if (!c.down) SPT_CUDA(cudaStreamCreateWithFlags(&c.down, cudaStreamNonBlocking));
    cs = &c;
    return SPT_OK;
}

struct Plan {
    int nfac = 0;                  // factors to upload, in upload order
    int fac_order[SPT_MAX_ORDER];  // mode of the k-th upload
    size_t fac_off[SPT_MAX_ORDER];
    size_t out_off[SPT_MAX_ORDER];
    size_t bytes = 0;
};

spt_status make_plan(spt_tensor t, int nmodes, const int *modes, spt_dtype fdt, int rank, int ld, Plan &pl) {
    if (!t || (nmodes > 0 && !modes)) return fail(SPT_EINVAL, "mttkrp_from_host: NULL argument");
    if (nmodes < 1 || nmodes > t->d) return fail(SPT_EINVAL, "mttkrp_from_host: nmodes must be in [1, order]");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16 && fdt != SPT_F64)
        return fail(SPT_EINVAL, "mttkrp_from_host: bad dtype");
    if (rank < 1 || ld < rank || ld % 8) return fail(SPT_EINVAL, "mttkrp_from_host: bad rank or ld");
    bool seen[SPT_MAX_ORDER] = {false}, queued[SPT_MAX_ORDER] = {false};
    for (int q = 0; q < nmodes; ++q) {
        if (modes[q] < 0 || modes[q] >= t->d) return fail(SPT_EINVAL, "mttkrp_from_host: mode out of range");
        if (seen[modes[q]]) return fail(SPT_EINVAL, "mttkrp_from_host: a mode is listed twice");
        seen[modes[q]] = true;
    }
    // uploads in order of first need: every factor but modes[0]'s, then the rest
    pl = Plan{};
    for (int q = 0; q < nmodes; ++q)
        for (int m = 0; m < t->d; ++m)
            if (m != modes[q] && !queued[m]) {
                queued[m] = true;
                pl.fac_order[pl.nfac++] = m;
            }
    const size_t es = (size_t)elem_bytes(fdt), ab = (size_t)acc_bytes(fdt);
    size_t off = 0;
    for (int k = 0; k < pl.nfac; ++k) {
        const int m = pl.fac_order[k];
        pl.fac_off[m] = off;
        off += round_up((size_t)t->dims[m] * ld * es);
    }
    for (int q = 0; q < nmodes; ++q) {
        pl.out_off[q] = off;
        off += round_up((size_t)t->dims[modes[q]] * ld * ab);
    }
    pl.bytes = off;
    return SPT_OK;
}

}  // namespace
}  // namespace spt

using namespace spt;

extern "C" {

spt_status mttkrp_from_host_workspace_size(spt_tensor t, int nmodes, const int *modes, spt_dtype fdt, int rank,
                                           int ld, size_t *bytes) {
    if (!bytes) return fail(SPT_EINVAL, "mttkrp_from_host_workspace_size: NULL bytes");
    Plan pl;
    spt_status c = make_plan(t, nmodes, modes, fdt, rank, ld, pl);
    if (c) return c;
    *bytes = pl.bytes;
    return SPT_OK;
}

spt_status mttkrp_from_host(spt_tensor t, int nmodes, const int *modes, const void *const *factors, spt_dtype fdt,
                            int rank, int ld, const void *lambda, void *const *out, void *workspace,
                            size_t workspace_bytes, void *stream) {
    Plan pl;
    spt_status c = make_plan(t, nmodes, modes, fdt, rank, ld, pl);
    if (c) return c;
    if (!factors || !out) return fail(SPT_EINVAL, "mttkrp_from_host: NULL factors or out");
    for (int k = 0; k < pl.nfac; ++k)
        if (!factors[pl.fac_order[k]]) return fail(SPT_EINVAL, "mttkrp_from_host: a needed factor is NULL");
    for (int q = 0; q < nmodes; ++q)
        if (!out[q]) return fail(SPT_EINVAL, "mttkrp_from_host: an output pointer is NULL");
    if (!workspace || ((uintptr_t)workspace & (ALIGN - 1)) || workspace_bytes < pl.bytes)
        return fail(SPT_EINVAL, "mttkrp_from_host: workspace NULL, not 256-byte aligned or too small");
    CopyStreams *cs = nullptr;
    c = copy_streams(cs);
    if (c) return c;

    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    const size_t es = (size_t)elem_bytes(fdt), ab = (size_t)acc_bytes(fdt);
    // events: start, one per upload, one per kernel, end of downloads
    cudaEvent_t ev[2 + 2 * SPT_MAX_ORDER];
    int nev = 0;
    auto new_event = [&](cudaEvent_t &e) {
        cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r == cudaSuccess) ev[nev++] = e;
        return r;
    };
    cudaError_t e = cudaSuccess;
    cudaEvent_t e_start = nullptr, e_up[SPT_MAX_ORDER] = {nullptr}, e_done = nullptr;
    const void *dfac[SPT_MAX_ORDER] = {nullptr};
    bool waited[SPT_MAX_ORDER] = {false};
    bool on_copy_streams = false;  // work may have been queued on cs->up / cs->down
    do {
        // the workspace is free once the caller's earlier work on `stream` is done
        if ((e = new_event(e_start)) != cudaSuccess) break;
        if ((e = cudaEventRecord(e_start, st)) != cudaSuccess) break;
        on_copy_streams = true;
        if ((e = cudaStreamWaitEvent(cs->up, e_start, 0)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(cs->down, e_start, 0)) != cudaSuccess) break;
        for (int k = 0; k < pl.nfac && e == cudaSuccess; ++k) {
            const int m = pl.fac_order[k];
            dfac[m] = ws + pl.fac_off[m];
            e = cudaMemcpyAsync(ws + pl.fac_off[m], factors[m], (size_t)t->dims[m] * ld * es,
                                cudaMemcpyHostToDevice, cs->up);
            if (e == cudaSuccess) e = new_event(e_up[m]);
            if (e == cudaSuccess) e = cudaEventRecord(e_up[m], cs->up);
        }
        if (e != cudaSuccess) break;
        for (int q = 0; q < nmodes; ++q) {
            const int n = modes[q];
            for (int m = 0; m < t->d && e == cudaSuccess; ++m)
                if (m != n && !waited[m]) {
                    waited[m] = true;
                    e = cudaStreamWaitEvent(st, e_up[m], 0);
                }
            if (e != cudaSuccess) break;
            c = mttkrp(t, n, dfac, fdt, rank, ld, lambda, ws + pl.out_off[q], nullptr, stream);
            if (c) break;
            cudaEvent_t e_k = nullptr;
            if ((e = new_event(e_k)) != cudaSuccess) break;
            if ((e = cudaEventRecord(e_k, st)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(cs->down, e_k, 0)) != cudaSuccess) break;
            e = cudaMemcpyAsync(out[q], ws + pl.out_off[q], (size_t)t->dims[n] * ld * ab, cudaMemcpyDeviceToHost,
                                cs->down);
            if (e != cudaSuccess) break;
        }
        if (c || e != cudaSuccess) break;
        // `stream` completes only after every download
        if ((e = new_event(e_done)) != cudaSuccess) break;
        if ((e = cudaEventRecord(e_done, cs->down)) != cudaSuccess) break;
        e = cudaStreamWaitEvent(st, e_done, 0);
    } while (false);
    if ((c || e != cudaSuccess) && on_copy_streams) {
        // a failed call still leaves `stream` ordered after every copy it
        // queued, so the caller may free or reuse the workspace and the host
        // buffers once `stream` is done; if the join cannot be enqueued, wait
        // for the copy streams here
        for (cudaStream_t cst : {cs->up, cs->down}) {
            cudaEvent_t j = nullptr;
            bool joined = cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess &&
                          cudaEventRecord(j, cst) == cudaSuccess && cudaStreamWaitEvent(st, j, 0) == cudaSuccess;
            if (j) cudaEventDestroy(j);
            if (!joined) cudaStreamSynchronize(cst);
        }
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);  // released once their work completes
    if (c) return c;
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp_from_host");
    return SPT_OK;
}

}  // extern "C"

// api.cu -- C-ABI entry points: errors, tensor ingest (Sec. 3 COO), mode
// permutations (Sec. 6), the MTTKRP call (Sec. 3 eq. mttkrp) and utilities.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace spt {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

spt_status fail(spt_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

spt_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return SPT_ECUDA;
}

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

size_t seg_bytes(int64_t n, size_t elem) {
    size_t b = (size_t)std::max<int64_t>(n, 1) * elem;
    return (b + 255) / 256 * 256;
}

namespace {
struct IdxSet {
    const int32_t *p[SPT_MAX_ORDER];
    int32_t dim[SPT_MAX_ORDER];
};

__global__ void range_check_kernel(IdxSet s, int d, int64_t n, unsigned long long *bad) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int m = 0; m < d; ++m) {
            const int32_t v = s.p[m][i];
            c += (v < 0 || v >= s.dim[m]);
        }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

// Shard of a tensor: nonzero i of the shard is nonzero perm[begin + i] of t.
__global__ void shard_gather_kernel(IdxSet src, const float *vals, const int32_t *perm, int64_t begin, int64_t n,
                                    int d, IdxSet dst_idx, float *dst_vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = perm[begin + i];
        for (int m = 0; m < d; ++m) const_cast<int32_t *>(dst_idx.p[m])[i] = src.p[m][q];
        dst_vals[i] = vals[q];
    }
}

spt_status free_tensor_buffers(spt_tensor t) {
    cudaStream_t st = 0;
    for (int n = 0; n < SPT_MAX_ORDER; ++n) {
        dfree(t->perm[n], st);
        dfree(t->sorted_buf[n], st);
        dfree(t->blk_buf[n], st);
    }
    dfree(t->coo_buf, st);
    dfree(t->dev_err, st);
    dfree(t->hot_buf, st);
    dfree(t->srec, st);
    cudaError_t e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? SPT_OK : cuda_fail(e, "tensor_destroy");
}
}  // namespace

}  // namespace spt

using namespace spt;

extern "C" {

const char *spt_last_error(void) { return g_err.c_str(); }

spt_status spt_device_info(int *sm, int *arch) {
    if (sm) *sm = sm_count();
    if (arch) *arch = 103;
    return SPT_OK;
}

spt_status tensor_create_coo(int order, const int64_t *dims, int64_t nnz,
                             const int32_t *const *idx, const float *vals, int flags,
                             void *stream, spt_tensor *out) {
    g_err.clear();
    if (!out) return fail(SPT_EINVAL, "tensor_create_coo: out is NULL");
    *out = nullptr;
    if (order < 1 || order > SPT_MAX_ORDER)
        return fail(SPT_EINVAL, "tensor_create_coo: order must be in [1, 8]");
    if (!dims) return fail(SPT_EINVAL, "tensor_create_coo: dims is NULL");
    for (int m = 0; m < order; ++m)
        if (dims[m] < 1 || dims[m] > INT32_MAX)
            return fail(SPT_EINVAL, "tensor_create_coo: every mode length must be in [1, 2^31-1]");
    if (nnz < 0 || nnz > INT32_MAX - 4096)
        return fail(SPT_EINVAL, "tensor_create_coo: nnz must be in [0, 2^31 - 4097]");
    if (flags & ~(SPT_DEVICE_PTRS | SPT_COALESCE))
        return fail(SPT_EINVAL, "tensor_create_coo: unknown flag bits");
    if (nnz > 0) {
        if (!idx || !vals) return fail(SPT_EINVAL, "tensor_create_coo: idx or vals is NULL");
        for (int m = 0; m < order; ++m)
            if (!idx[m]) return fail(SPT_EINVAL, "tensor_create_coo: idx[m] is NULL");
    }
    cudaStream_t st = (cudaStream_t)stream;
    spt_tensor t = new (std::nothrow) spt_tensor_s();
    if (!t) return fail(SPT_ENOMEM, "tensor_create_coo: host allocation failed");
    cudaGetDevice(&t->device);
    t->d = order;
    for (int m = 0; m < order; ++m) t->dims[m] = dims[m];
    t->nnz = nnz;
    const size_t seg = seg_bytes(nnz, 4);
    spt_status s = dmalloc(&t->coo_buf, seg * (order + 1), st);
    if (!s) s = dmalloc((void **)&t->dev_err, sizeof(int), st);
    if (s) { free_tensor_buffers(t); delete t; return s; }
    for (int m = 0; m < order; ++m) t->idx[m] = reinterpret_cast<int32_t *>((char *)t->coo_buf + seg * m);
    t->vals = reinterpret_cast<float *>((char *)t->coo_buf + seg * order);
    cudaError_t e = cudaMemsetAsync(t->dev_err, 0, sizeof(int), st);
    const cudaMemcpyKind kind = (flags & SPT_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int m = 0; m < order && e == cudaSuccess && nnz > 0; ++m)
        e = cudaMemcpyAsync(t->idx[m], idx[m], 4 * nnz, kind, st);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(t->vals, vals, 4 * nnz, kind, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s = cuda_fail(e, "tensor_create_coo: copy of the nonzeros");
        free_tensor_buffers(t);
        delete t;
        return s;
    }
    // coordinate range check on the device
    unsigned long long *bad = nullptr;
    s = dmalloc((void **)&bad, sizeof(unsigned long long), st);
    if (s) { free_tensor_buffers(t); delete t; return s; }
    cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
    if (nnz > 0) {
        IdxSet is;
        for (int m = 0; m < order; ++m) { is.p[m] = t->idx[m]; is.dim[m] = (int32_t)dims[m]; }
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nnz + 255) / 256, sm_count() * 8));
        range_check_kernel<<<grid, 256, 0, st>>>(is, order, nnz, bad);
    }
    unsigned long long nbad = 0;
    cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, st);
    dfree(bad, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        s = cuda_fail(e, "tensor_create_coo: range check");
        free_tensor_buffers(t);
        delete t;
        return s;
    }
    if (nbad) {
        free_tensor_buffers(t);
        delete t;
        return fail(SPT_ERANGE, "tensor_create_coo: " + std::to_string(nbad) +
                                    " coordinate(s) outside [0, I_m)");
    }
    if (flags & SPT_COALESCE) {
        s = coalesce_tensor(t, st);
        if (s) { free_tensor_buffers(t); delete t; return s; }
    }
    s = build_hot_rows(t, st);
    if (s) { free_tensor_buffers(t); delete t; return s; }
    *out = t;
    return SPT_OK;
}

spt_status tensor_create_shard(spt_tensor t, int mode, int64_t begin, int64_t end, void *stream, spt_tensor *out) {
    if (!t || !out) return fail(SPT_EINVAL, "tensor_create_shard: NULL argument");
    *out = nullptr;
    if (mode < 0 || mode >= t->d) return fail(SPT_EINVAL, "tensor_create_shard: mode out of range");
    if (begin < 0 || end < begin || end > t->nnz)
        return fail(SPT_EINVAL, "tensor_create_shard: need 0 <= begin <= end <= nnz");
    if (!t->perm[mode]) return fail(SPT_ESTATE, "tensor_create_shard: needs build_mode_permutation(mode)");
    cudaStream_t st = (cudaStream_t)stream;
    spt_tensor s = new (std::nothrow) spt_tensor_s();
    if (!s) return fail(SPT_ENOMEM, "tensor_create_shard: host allocation failed");
    cudaGetDevice(&s->device);
    s->d = t->d;
    for (int m = 0; m < t->d; ++m) s->dims[m] = t->dims[m];
    const int64_t n = end - begin;
    s->nnz = n;
    const size_t seg = seg_bytes(n, 4);
    spt_status c = dmalloc(&s->coo_buf, seg * (t->d + 1), st);
    if (!c) c = dmalloc((void **)&s->dev_err, sizeof(int), st);
    if (c) { free_tensor_buffers(s); delete s; return c; }
    IdxSet src, dst;
    for (int m = 0; m < t->d; ++m) {
        s->idx[m] = reinterpret_cast<int32_t *>((char *)s->coo_buf + seg * m);
        src.p[m] = t->idx[m];
        dst.p[m] = s->idx[m];
    }
    s->vals = reinterpret_cast<float *>((char *)s->coo_buf + seg * t->d);
    cudaError_t e = cudaMemsetAsync(s->dev_err, 0, sizeof(int), st);
    if (e == cudaSuccess && n > 0) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8));
        shard_gather_kernel<<<grid, 256, 0, st>>>(src, t->vals, t->perm[mode], begin, n, t->d, dst, s->vals);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        c = cuda_fail(e, "tensor_create_shard");
        free_tensor_buffers(s);
        delete s;
        return c;
    }
    // a subset of distinct coordinates is coalesced too; its ||X||^2 is its own
    s->coalesced = t->coalesced;
    c = s->coalesced ? compute_norm2(s, st) : SPT_OK;
    if (!c) c = build_hot_rows(s, st);
    if (c) { free_tensor_buffers(s); delete s; return c; }
    *out = s;
    return SPT_OK;
}

spt_status tensor_destroy(spt_tensor t) {
    if (!t) return fail(SPT_EINVAL, "tensor_destroy: NULL tensor");
    drop_graphs(t);
    spt_status s = free_tensor_buffers(t);
    delete t;
    return s;
}

spt_status tensor_info(spt_tensor t, int *order, int64_t *dims, int64_t *nnz, int *flags) {
    if (!t) return fail(SPT_EINVAL, "tensor_info: NULL tensor");
    if (order) *order = t->d;
    if (dims)
        for (int m = 0; m < SPT_MAX_ORDER; ++m) dims[m] = m < t->d ? t->dims[m] : 0;
    if (nnz) *nnz = t->nnz;
    if (flags) *flags = t->coalesced ? SPT_COALESCE : 0;
    return SPT_OK;
}

spt_status tensor_get_coo(spt_tensor t, int32_t *const *idx, float *vals, void *stream) {
    if (!t) return fail(SPT_EINVAL, "tensor_get_coo: NULL tensor");
    cudaStream_t st = (cudaStream_t)stream;
    if (t->nnz == 0) return SPT_OK;
    for (int m = 0; m < t->d; ++m)
        if (idx && idx[m])
            SPT_CUDA(cudaMemcpyAsync(idx[m], t->idx[m], 4 * t->nnz, cudaMemcpyDeviceToDevice, st));
    if (vals) SPT_CUDA(cudaMemcpyAsync(vals, t->vals, 4 * t->nnz, cudaMemcpyDeviceToDevice, st));
    return SPT_OK;
}

spt_status tensor_norm2(spt_tensor t, double *out) {
    if (!t || !out) return fail(SPT_EINVAL, "tensor_norm2: NULL argument");
    if (!t->coalesced) return fail(SPT_ESTATE, "tensor_norm2: tensor is not coalesced");
    *out = t->xnorm2;
    return SPT_OK;
}

spt_status build_mode_permutation(spt_tensor t, int mode, int flags, void *stream) {
    if (!t) return fail(SPT_EINVAL, "build_mode_permutation: NULL tensor");
    if (mode < -1 || mode >= t->d) return fail(SPT_EINVAL, "build_mode_permutation: bad mode");
    if (flags & ~(SPT_PERM_INDEX_ONLY | SPT_PERM_SLICE_ORDER))
        return fail(SPT_EINVAL, "build_mode_permutation: unknown flag bits");
    cudaStream_t st = (cudaStream_t)stream;
    drop_graphs(t);
    for (int n = 0; n < t->d; ++n) {
        if (mode >= 0 && n != mode) continue;
        spt_status s = build_perm_mode(t, n, (flags & SPT_PERM_INDEX_ONLY) != 0, st, (flags & SPT_PERM_SLICE_ORDER) != 0);
        if (s) return s;
    }
    return SPT_OK;
}

spt_status tensor_storage_records(spt_tensor t, int keep, void *stream) {
    if (!t) return fail(SPT_EINVAL, "tensor_storage_records: NULL tensor");
    if (keep != 0 && keep != 1) return fail(SPT_EINVAL, "tensor_storage_records: keep must be 0 or 1");
    cudaStream_t st = (cudaStream_t)stream;
    drop_graphs(t);
    if (!keep) {
        dfree(t->srec, st);
        t->srec = nullptr;
        return SPT_OK;
    }
    return t->srec ? SPT_OK : build_storage_records(t, st);
}

spt_status build_mode_l2_blocks(spt_tensor t, int mode, int blocked_mode, int64_t block_rows, void *stream) {
    if (!t) return fail(SPT_EINVAL, "build_mode_l2_blocks: NULL tensor");
    if (mode < 0 || mode >= t->d) return fail(SPT_EINVAL, "build_mode_l2_blocks: bad mode");
    cudaStream_t st = (cudaStream_t)stream;
    if (block_rows == 0) {  // drop
        drop_graphs(t);
        if (t->blk_buf[mode]) dfree(t->blk_buf[mode], st);
        t->blk_buf[mode] = nullptr;
        t->blk_off[mode].clear();
        t->blk_mode[mode] = -1;
        t->blk_rows[mode] = 0;
        SPT_CUDA(cudaStreamSynchronize(st));
        return SPT_OK;
    }
    if (!t->sorted_buf[mode])
        return fail(SPT_ESTATE, "build_mode_l2_blocks: needs the mode-sorted copy (build_mode_permutation)");
    int bm = blocked_mode;
    if (bm == -1) {
        for (int m = 0; m < t->d; ++m)
            if (m != mode && (bm < 0 || t->dims[m] > t->dims[bm])) bm = m;
    }
    if (bm < 0 || bm >= t->d || bm == mode) return fail(SPT_EINVAL, "build_mode_l2_blocks: bad blocked mode");
    const int64_t rows = block_rows < 0 ? SPT_L2_BLOCK_ROWS_DEFAULT : block_rows;
    if ((t->dims[bm] + rows - 1) / rows > 65536)
        return fail(SPT_EINVAL, "build_mode_l2_blocks: more than 65536 blocks");
    drop_graphs(t);
    return build_l2_blocks(t, mode, bm, rows, st);
}

spt_status tensor_l2_blocks(spt_tensor t, int mode, int *blocked_mode, int64_t *block_rows, int64_t *groups) {
    if (!t) return fail(SPT_EINVAL, "tensor_l2_blocks: NULL tensor");
    if (mode < 0 || mode >= t->d) return fail(SPT_EINVAL, "tensor_l2_blocks: bad mode");
    if (blocked_mode) *blocked_mode = t->blk_buf[mode] ? t->blk_mode[mode] : -1;
    if (block_rows) *block_rows = t->blk_buf[mode] ? t->blk_rows[mode] : 0;
    if (groups) *groups = t->blk_buf[mode] ? (int64_t)t->blk_off[mode].size() - 1 : 0;
    return SPT_OK;
}

spt_status tensor_get_permutation(spt_tensor t, int mode, int32_t *perm, void *stream) {
    if (!t || !perm) return fail(SPT_EINVAL, "tensor_get_permutation: NULL argument");
    if (mode < 0 || mode >= t->d) return fail(SPT_EINVAL, "tensor_get_permutation: bad mode");
    if (!t->perm[mode]) return fail(SPT_ESTATE, "tensor_get_permutation: permutation not built");
    if (t->nnz)
        SPT_CUDA(cudaMemcpyAsync(perm, t->perm[mode], 4 * t->nnz, cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
    return SPT_OK;
}

spt_status tensor_check(spt_tensor t, void *stream) {
    if (!t) return fail(SPT_EINVAL, "tensor_check: NULL tensor");
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    SPT_CUDA(cudaMemcpyAsync(&h, t->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPT_CUDA(cudaStreamSynchronize(st));
    if (h) {  // reported once: clear the word for the calls that follow
        SPT_CUDA(cudaMemsetAsync(t->dev_err, 0, sizeof(int), st));
        SPT_CUDA(cudaStreamSynchronize(st));
    }
    if (h == SPT_DEV_TIMEOUT) return fail(SPT_ETIMEOUT, "a bounded device wait ran out");
    if (h) return fail(SPT_ECUDA, "device status word " + std::to_string(h));
    return SPT_OK;
}

static spt_status mttkrp_impl(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank,
                              int ld, const void *lambda, void *out, const spt_schedule *sched,
                              void *stream, bool det) {
    if (!t) return fail(SPT_EINVAL, "mttkrp: NULL tensor");
    if (mode < 0 || mode >= t->d) return fail(SPT_EINVAL, "mttkrp: mode out of range");
    if (t->d > SPT_MAX_KERNEL_ORDER) return fail(SPT_EUNSUPPORTED, "mttkrp: order > 5");
    if (fdt != SPT_F32 && fdt != SPT_BF16 && fdt != SPT_F16 && fdt != SPT_F64)
        return fail(SPT_EINVAL, "mttkrp: bad dtype");
    if (rank < 1) return fail(SPT_EINVAL, "mttkrp: rank must be >= 1");
    if (ld < rank || ld % 8) return fail(SPT_EINVAL, "mttkrp: ld must be >= rank and a multiple of 8");
    if (ld > (1 << 28)) return fail(SPT_EUNSUPPORTED, "mttkrp: ld above 2^28 elements");
    if (!out || ((uintptr_t)out & 15)) return fail(SPT_EINVAL, "mttkrp: out NULL or not 16-byte aligned");
    if (lambda && ((uintptr_t)lambda & (acc_bytes(fdt) - 1)))
        return fail(SPT_EINVAL, "mttkrp: lambda not aligned to its element");
    if (t->d > 1 && !factors) return fail(SPT_EINVAL, "mttkrp: factors is NULL");
    for (int m = 0; m < t->d; ++m) {
        if (m == mode) continue;
        if (!factors[m] || ((uintptr_t)factors[m] & 15))
            return fail(SPT_EINVAL, "mttkrp: a factor pointer is NULL or not 16-byte aligned");
    }
    spt_schedule s = sched ? *sched : default_schedule(t, mode, fdt, rank);
    if (s.scatter == SPT_SCATTER_AUTO) s.scatter = default_schedule(t, mode, fdt, rank).scatter;
    if (det) {
        if (!t->sorted_buf[mode])
            return fail(SPT_ESTATE, "mttkrp_deterministic: needs the mode-sorted copy (build_mode_permutation)");
        if (rank > 256) return fail(SPT_EUNSUPPORTED, "mttkrp_deterministic: rank must be <= 256");
        if (!sched) {  // a recorded schedule of another kind: keep its sizes where they fit
            s.scatter = SPT_SCATTER_SORTED;
            if (s.lanes_per_nnz * s.chunks * 4 < rank) {
                s.lanes_per_nnz = 32;
                s.chunks = rank > 128 ? 2 : 1;
            }
        }
        if (s.scatter != SPT_SCATTER_SORTED || s.lanes_per_nnz * s.chunks * 4 < rank)
            return fail(SPT_EINVAL, "mttkrp_deterministic: the schedule must be sorted with lanes x chunks x 4 >= rank");
    }
    spt_status c = check_schedule(t, mode, fdt, rank, s);
    if (c) return c;
    return launch_mttkrp(t, mode, factors, fdt, rank, ld, lambda, out, s, (cudaStream_t)stream, nullptr, det);
}

spt_status mttkrp(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank,
                  int ld, const void *lambda, void *out, const spt_schedule *sched,
                  void *stream) {
    return mttkrp_impl(t, mode, factors, fdt, rank, ld, lambda, out, sched, stream, false);
}

spt_status mttkrp_deterministic(spt_tensor t, int mode, const void *const *factors, spt_dtype fdt, int rank,
                                int ld, const void *lambda, void *out, const spt_schedule *sched,
                                void *stream) {
    return mttkrp_impl(t, mode, factors, fdt, rank, ld, lambda, out, sched, stream, true);
}

spt_status tensor_set_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank, const spt_schedule *s) {
    if (!t) return fail(SPT_EINVAL, "tensor_set_schedule: NULL tensor");
    if (mode < 0 || mode >= t->d || rank < 1) return fail(SPT_EINVAL, "tensor_set_schedule: bad mode/rank");
    drop_graphs(t);
    if (!s) { t->pref_set[mode] = false; return SPT_OK; }
    spt_status c = check_schedule(t, mode, fdt, rank, *s);
    if (c) return c;
    t->pref_set[mode] = true;
    t->pref_rank[mode] = rank;
    t->pref_fdt[mode] = fdt;
    t->pref[mode] = *s;
    return SPT_OK;
}

spt_status mttkrp_default_schedule(spt_tensor t, int mode, spt_dtype fdt, int rank,
                                   spt_schedule *out) {
    if (!t || !out) return fail(SPT_EINVAL, "mttkrp_default_schedule: NULL argument");
    if (mode < 0 || mode >= t->d || rank < 1) return fail(SPT_EINVAL, "mttkrp_default_schedule: bad mode/rank");
    *out = default_schedule(t, mode, fdt, rank);
    return SPT_OK;
}

// Tab. "sizes" (Sec. 5): GPU vector_size and factor block size FBS by rank.
spt_status mttkrp_paper_sizes(int R, int *vector_size, int *fbs) {
    if (R < 1) return fail(SPT_EINVAL, "mttkrp_paper_sizes: rank must be >= 1");
    int vs, fb;
    if (R == 1) { vs = 1; fb = 1; }
    else if (R == 2) { vs = 2; fb = 2; }
    else if (R == 3) { vs = 2; fb = 4; }
    else if (R == 4) { vs = 4; fb = 4; }
    else if (R <= 7) { vs = 4; fb = 8; }
    else if (R == 8) { vs = 8; fb = 8; }
    else if (R <= 16) { vs = 8; fb = 16; }
    else if (R <= 24) { vs = 8; fb = 24; }
    else if (R <= 47) { vs = 8; fb = 32; }
    else if (R == 48) { vs = 16; fb = 48; }
    else if (R <= 95) { vs = 16; fb = 64; }
    else if (R == 96) { vs = 32; fb = 96; }
    else { vs = 32; fb = 128; }
    if (vector_size) *vector_size = vs;
    if (fbs) *fbs = fb;
    return SPT_OK;
}

// The Tab. "sizes" rule on this kernel: the rank block (the paper's FBS) is
// covered by lanes * chunks 16-byte chunks; NZPTM = 128 nonzeros per group;
// a team of 128 threads = 4 warps.
spt_status mttkrp_paper_schedule(int rank, spt_dtype fdt, int scatter, spt_schedule *out) {
    if (!out) return fail(SPT_EINVAL, "mttkrp_paper_schedule: NULL out");
    int vs = 0, fbs = 0;
    spt_status s = mttkrp_paper_sizes(rank, &vs, &fbs);
    if (s) return s;
    const int vec = 4;  // columns per lane chunk
    (void)fdt;
    int need = (fbs + vec - 1) / vec;
    int lanes = 1;
    while (lanes < need && lanes < 32) lanes <<= 1;
    out->scatter = scatter;
    out->lanes_per_nnz = lanes;
    out->chunks = need > 32 ? 2 : 1;
    out->nnz_per_group = 128;
    out->warps_per_cta = 4;
    out->ctas_per_sm = 0;
    return SPT_OK;
}

}  // extern "C"

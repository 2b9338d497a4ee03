"""ctypes binding of ``libspt.so`` -- argument marshalling only.

Each function has the name of the C entry point it calls (declared in
``include/spt.h``) and takes plain integers for device pointers (for example
``torch_tensor.data_ptr()``) and CUDA streams (``torch.cuda.current_stream()
.cuda_stream``).  A non-zero status raises :class:`SptError`.  There is no
fallback: if the compiled library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspt.so")

SPT_OK, SPT_EINVAL, SPT_ERANGE, SPT_ENOMEM, SPT_ECUDA = 0, 1, 2, 3, 4
SPT_EUNSUPPORTED, SPT_ESINGULAR, SPT_ETIMEOUT, SPT_ESTATE = 5, 6, 7, 8
SPT_F32, SPT_BF16, SPT_F16, SPT_F64 = 0, 1, 2, 3
SPT_DEVICE_PTRS, SPT_COALESCE = 1, 2
SPT_PERM_INDEX_ONLY, SPT_PERM_SLICE_ORDER = 1, 2
SPT_SCATTER_AUTO, SPT_SCATTER_ATOMIC, SPT_SCATTER_PERM, SPT_SCATTER_SORTED, SPT_SCATTER_PRIVATE = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "SPT_OK", 1: "SPT_EINVAL", 2: "SPT_ERANGE", 3: "SPT_ENOMEM", 4: "SPT_ECUDA",
                5: "SPT_EUNSUPPORTED", 6: "SPT_ESINGULAR", 7: "SPT_ETIMEOUT", 8: "SPT_ESTATE"}
DTYPES = {"f32": SPT_F32, "bf16": SPT_BF16, "f16": SPT_F16, "f64": SPT_F64}
SCATTERS = {"auto": SPT_SCATTER_AUTO, "atomic": SPT_SCATTER_ATOMIC, "perm": SPT_SCATTER_PERM,
            "sorted": SPT_SCATTER_SORTED, "private": SPT_SCATTER_PRIVATE}


class SptError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class spt_schedule(C.Structure):
    _fields_ = [("scatter", C.c_int32), ("lanes_per_nnz", C.c_int32), ("chunks", C.c_int32),
                ("nnz_per_group", C.c_int32), ("warps_per_cta", C.c_int32),
                ("ctas_per_sm", C.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}

    @classmethod
    def make(cls, scatter=SPT_SCATTER_AUTO, lanes_per_nnz=4, chunks=1, nnz_per_group=32,
             warps_per_cta=8, ctas_per_sm=0):
        if isinstance(scatter, str):
            scatter = SCATTERS[scatter]
        return cls(scatter, lanes_per_nnz, chunks, nnz_per_group, warps_per_cta, ctas_per_sm)


class spt_selector(C.Structure):
    _fields_ = [("F", C.c_int), ("H1", C.c_int), ("H2", C.c_int), ("K", C.c_int),
                ("params", C.c_void_p), ("mean", C.POINTER(C.c_float)),
                ("std", C.POINTER(C.c_float)), ("anchor_margin", C.c_float)]


class spt_batch_item(C.Structure):
    _fields_ = [("tensor", C.c_void_p), ("mode", C.c_int), ("rank", C.c_int), ("ld", C.c_int),
                ("factors", C.POINTER(C.c_void_p)), ("outs", C.POINTER(C.c_void_p)),
                ("scheds", C.POINTER(spt_schedule))]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run paper_1809_09175_gb300/build.py (or "
                      "__graft_entry__.build()) to compile the CUDA library")

_L = C.CDLL(LIB_PATH)
_vp = C.c_void_p
_i64p = C.POINTER(C.c_int64)


def _sig(name, *args):
    f = getattr(_L, name)
    f.argtypes = list(args)
    f.restype = C.c_int
    return f


_L.spt_last_error.restype = C.c_char_p
_L.spt_last_error.argtypes = []
_sig("spt_device_info", C.POINTER(C.c_int), C.POINTER(C.c_int))
_sig("tensor_create_coo", C.c_int, _i64p, C.c_int64, C.POINTER(_vp), _vp, C.c_int, _vp,
     C.POINTER(_vp))
_sig("tensor_destroy", _vp)
_sig("tensor_info", _vp, C.POINTER(C.c_int), _i64p, _i64p, C.POINTER(C.c_int))
_sig("tensor_get_coo", _vp, C.POINTER(_vp), _vp, _vp)
_sig("tensor_norm2", _vp, C.POINTER(C.c_double))
_sig("tensor_check", _vp, _vp)
_sig("build_mode_permutation", _vp, C.c_int, C.c_int, _vp)
_sig("tensor_get_permutation", _vp, C.c_int, _vp, _vp)
_sig("mttkrp", _vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _vp, _vp,
     C.POINTER(spt_schedule), _vp)
_sig("mttkrp_deterministic", _vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _vp, _vp,
     C.POINTER(spt_schedule), _vp)
_sig("mttkrp_from_host_workspace_size", _vp, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int,
     C.POINTER(C.c_size_t))
_sig("mttkrp_from_host", _vp, C.c_int, C.POINTER(C.c_int), C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _vp,
     C.POINTER(_vp), _vp, C.c_size_t, _vp)
_sig("mttkrp_default_schedule", _vp, C.c_int, C.c_int, C.c_int, C.POINTER(spt_schedule))
_sig("tensor_set_schedule", _vp, C.c_int, C.c_int, C.c_int, C.POINTER(spt_schedule))
_sig("mttkrp_paper_sizes", C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int))
_sig("mttkrp_paper_schedule", C.c_int, C.c_int, C.c_int, C.POINTER(spt_schedule))
_sig("spt_stream_copy", _vp, _vp, C.c_size_t, _vp)
_sig("spt_convert_f32", _vp, _vp, C.c_int, C.c_int64, _vp)
_sig("spt_fma_probe", C.c_int, C.c_int64, _vp, C.POINTER(C.c_double), _vp)

EXPORTED = ["spt_last_error", "spt_device_info", "tensor_create_coo", "tensor_destroy",
            "tensor_info", "tensor_get_coo", "tensor_norm2", "tensor_check",
            "build_mode_permutation", "tensor_get_permutation", "mttkrp", "mttkrp_deterministic",
            "mttkrp_from_host_workspace_size", "mttkrp_from_host",
            "mttkrp_default_schedule", "tensor_set_schedule", "mttkrp_paper_sizes", "mttkrp_paper_schedule",
            "spt_stream_copy", "spt_convert_f32", "spt_fma_probe"]


def _try_sig(name, *args):
    if hasattr(_L, name):
        _sig(name, *args)
        EXPORTED.append(name)


# CP-ALS and later entry points (declared when present in the library)
_try_sig("cp_als_workspace_size", _vp, C.c_int, C.c_int, C.POINTER(C.c_size_t))
_try_sig("cp_als_step", _vp, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _vp, _vp, _vp,
         C.c_size_t, _vp)
_try_sig("cp_als_status", _vp, _vp)
_try_sig("mode_permutation_noalloc", _vp, C.c_int64, C.c_int64, _vp, _vp)
_try_sig("gcp_gradient", _vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp)
SPT_LOSS_POISSON, SPT_LOSS_BERNOULLI_LOGIT, SPT_LOSS_GAUSSIAN = 0, 1, 2
LOSSES = {"poisson": SPT_LOSS_POISSON, "bernoulli": SPT_LOSS_BERNOULLI_LOGIT, "gaussian": SPT_LOSS_GAUSSIAN}
SPT_NUM_CANDIDATES, SPT_NUM_FEATURES = 48, 12
_fp = C.POINTER(C.c_float)
_try_sig("mttkrp_candidates", _vp, C.c_int, C.c_int, C.POINTER(spt_schedule), C.POINTER(C.c_int))
_try_sig("mttkrp_time_schedule", _vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _vp,
         C.POINTER(spt_schedule), C.c_int, _fp, _vp)
_try_sig("mttkrp_autotune", _vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _vp, C.c_int,
         C.POINTER(spt_schedule), _fp, _fp, _vp)
_try_sig("tensor_mode_features", _vp, C.c_int, C.c_int, C.c_int, _fp)
_try_sig("mlp_forward", C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp)
_try_sig("mlp_loss_grad", C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp,
         _vp, _vp, _vp)
_try_sig("mlp_adam", C.c_int64, _vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_float,
         C.c_int, _vp)
_try_sig("mlp_infer", C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp)
_try_sig("mttkrp_select", _vp, C.c_int, C.c_int, C.c_int, C.POINTER(spt_selector),
         C.POINTER(spt_schedule), _fp, _vp)
for _n in ("mlp_param_count", "mlp_workspace_floats"):
    getattr(_L, _n).restype = C.c_int64
_L.mlp_param_count.argtypes = [C.c_int] * 4
_L.mlp_workspace_floats.argtypes = [C.c_int] * 5
EXPORTED += ["mlp_param_count", "mlp_workspace_floats"]
_try_sig("mttkrp_batch_create", C.c_int, C.POINTER(spt_batch_item), C.c_int, C.POINTER(_vp))
_try_sig("mttkrp_batch_run", _vp, _vp)
_try_sig("mttkrp_batch_info", _vp, _i64p, _i64p, C.POINTER(C.c_int))
_try_sig("mttkrp_batch_check", _vp, _vp)
_try_sig("mttkrp_batch_destroy", _vp)
_try_sig("spt_set_wait_tries", C.c_int64)
_try_sig("spt_row_gather_probe", C.c_int, _vp, C.c_int64, _vp, C.c_int64, _vp, _vp, C.c_int64, _vp, _vp, _vp)
_try_sig("tensor_create_shard", _vp, C.c_int, C.c_int64, C.c_int64, _vp, C.POINTER(_vp))
_try_sig("tensor_storage_records", _vp, C.c_int, _vp)
_try_sig("build_mode_l2_blocks", _vp, C.c_int, C.c_int, C.c_int64, _vp)
_try_sig("tensor_l2_blocks", _vp, C.c_int, C.POINTER(C.c_int), _i64p, _i64p)
_try_sig("cp_als_hinv", _vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp)
_try_sig("cp_als_apply", _vp, C.c_int64, C.c_int, C.c_int, _vp, _vp, _vp, _vp)
_try_sig("cp_als_normalize", _vp, _vp, C.c_int64, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp, _vp, _vp)
_try_sig("cp_als_gram", _vp, C.c_int64, C.c_int, C.c_int, C.c_int, _vp, _vp)
_try_sig("cp_als_fit", _vp, C.c_int, C.c_int, _vp, _vp, C.c_double, _vp, _vp)
SPT_NOALLOC_MAX_NNZ = 1835008


def lib():
    return _L


def _chk(st: int):
    if st != SPT_OK:
        raise SptError(st, _L.spt_last_error().decode())


def spt_last_error() -> str:
    return _L.spt_last_error().decode()


def _ptrs(ps: Sequence[Optional[int]]):
    return (_vp * len(ps))(*[p if p else None for p in ps])


def _dt(fdt):
    return DTYPES[fdt] if isinstance(fdt, str) else int(fdt)


def spt_device_info():
    sm, arch = C.c_int(), C.c_int()
    _chk(_L.spt_device_info(C.byref(sm), C.byref(arch)))
    return sm.value, arch.value


def tensor_create_coo(order: int, dims: Sequence[int], nnz: int, idx_ptrs: Sequence[int],
                      vals_ptr: int, flags: int = 0, stream: int = 0) -> int:
    """Returns the tensor handle (an integer)."""
    dims_a = (C.c_int64 * order)(*[int(x) for x in dims])
    out = _vp()
    _chk(_L.tensor_create_coo(order, dims_a, int(nnz), _ptrs(idx_ptrs), vals_ptr or None, flags,
                              stream or None, C.byref(out)))
    return out.value


def tensor_destroy(t: int):
    _chk(_L.tensor_destroy(t))


def tensor_info(t: int):
    order, flags = C.c_int(), C.c_int()
    dims = (C.c_int64 * 8)()
    nnz = C.c_int64()
    _chk(_L.tensor_info(t, C.byref(order), dims, C.byref(nnz), C.byref(flags)))
    return order.value, [int(dims[m]) for m in range(order.value)], nnz.value, flags.value


def tensor_get_coo(t: int, idx_ptrs: Sequence[Optional[int]], vals_ptr: Optional[int], stream: int = 0):
    _chk(_L.tensor_get_coo(t, _ptrs(idx_ptrs), vals_ptr or None, stream or None))


def tensor_norm2(t: int) -> float:
    v = C.c_double()
    _chk(_L.tensor_norm2(t, C.byref(v)))
    return v.value


def tensor_check(t: int, stream: int = 0):
    _chk(_L.tensor_check(t, stream or None))


def build_mode_permutation(t: int, mode: int = -1, flags: int = 0, stream: int = 0):
    _chk(_L.build_mode_permutation(t, mode, flags, stream or None))


def tensor_get_permutation(t: int, mode: int, perm_ptr: int, stream: int = 0):
    _chk(_L.tensor_get_permutation(t, mode, perm_ptr, stream or None))


def mttkrp(t: int, mode: int, factor_ptrs: Sequence[Optional[int]], fdt, rank: int, ld: int,
           lambda_ptr: Optional[int], out_ptr: int, sched: Optional[spt_schedule] = None,
           stream: int = 0):
    _chk(_L.mttkrp(t, mode, _ptrs(factor_ptrs), _dt(fdt), rank, ld, lambda_ptr or None, out_ptr,
                   C.byref(sched) if sched is not None else None, stream or None))


def mttkrp_deterministic(t: int, mode: int, factor_ptrs: Sequence[Optional[int]], fdt, rank: int, ld: int,
                         lambda_ptr: Optional[int], out_ptr: int, sched: Optional[spt_schedule] = None,
                         stream: int = 0):
    _chk(_L.mttkrp_deterministic(t, mode, _ptrs(factor_ptrs), _dt(fdt), rank, ld, lambda_ptr or None,
                                 out_ptr, C.byref(sched) if sched is not None else None, stream or None))


def mttkrp_from_host_workspace_size(t: int, modes: Sequence[int], fdt, rank: int, ld: int) -> int:
    m = (C.c_int * len(modes))(*modes)
    n = C.c_size_t()
    _chk(_L.mttkrp_from_host_workspace_size(t, len(modes), m, _dt(fdt), rank, ld, C.byref(n)))
    return n.value


def mttkrp_from_host(t: int, modes: Sequence[int], host_factor_ptrs: Sequence[Optional[int]], fdt, rank: int,
                     ld: int, lambda_ptr: Optional[int], host_out_ptrs: Sequence[int], ws_ptr: int,
                     ws_bytes: int, stream: int = 0):
    m = (C.c_int * len(modes))(*modes)
    outs = (_vp * len(host_out_ptrs))(*[p or None for p in host_out_ptrs])
    _chk(_L.mttkrp_from_host(t, len(modes), m, _ptrs(host_factor_ptrs), _dt(fdt), rank, ld, lambda_ptr or None,
                             outs, ws_ptr, ws_bytes, stream or None))


def mttkrp_default_schedule(t: int, mode: int, fdt, rank: int) -> spt_schedule:
    s = spt_schedule()
    _chk(_L.mttkrp_default_schedule(t, mode, _dt(fdt), rank, C.byref(s)))
    return s


def tensor_set_schedule(t: int, mode: int, fdt, rank: int, sched: Optional[spt_schedule]):
    _chk(_L.tensor_set_schedule(t, mode, _dt(fdt), rank, C.byref(sched) if sched is not None else None))


def mttkrp_paper_sizes(rank: int):
    vs, fbs = C.c_int(), C.c_int()
    _chk(_L.mttkrp_paper_sizes(rank, C.byref(vs), C.byref(fbs)))
    return vs.value, fbs.value


def mttkrp_paper_schedule(rank: int, fdt, scatter) -> spt_schedule:
    s = spt_schedule()
    sc = SCATTERS[scatter] if isinstance(scatter, str) else int(scatter)
    _chk(_L.mttkrp_paper_schedule(rank, _dt(fdt), sc, C.byref(s)))
    return s


def spt_stream_copy(src_ptr: int, dst_ptr: int, nbytes: int, stream: int = 0):
    _chk(_L.spt_stream_copy(src_ptr, dst_ptr, nbytes, stream or None))


def spt_convert_f32(src_ptr: int, dst_ptr: int, fdt, n: int, stream: int = 0):
    _chk(_L.spt_convert_f32(src_ptr, dst_ptr, _dt(fdt), n, stream or None))


def spt_fma_probe(fdt, iters: int, sink_ptr: int, stream: int = 0) -> float:
    """Enqueue the FMA-rate probe; returns the flops it performs."""
    v = C.c_double()
    _chk(_L.spt_fma_probe(_dt(fdt), iters, sink_ptr, C.byref(v), stream or None))
    return v.value


def cp_als_workspace_size(t: int, rank: int, ld: int) -> int:
    v = C.c_size_t()
    _chk(_L.cp_als_workspace_size(t, rank, ld, C.byref(v)))
    return v.value


def cp_als_step(t: int, factor_ptrs: Sequence[int], fdt, rank: int, ld: int, lambda_ptr: int,
                fit_ptr: Optional[int], workspace_ptr: int, workspace_bytes: int, stream: int = 0):
    _chk(_L.cp_als_step(t, _ptrs(factor_ptrs), _dt(fdt), rank, ld, lambda_ptr, fit_ptr or None,
                        workspace_ptr, workspace_bytes, stream or None))


def cp_als_status(workspace_ptr: int, stream: int = 0):
    _chk(_L.cp_als_status(workspace_ptr, stream or None))


def tensor_storage_records(t: int, keep: int = 1, stream: int = 0):
    _chk(_L.tensor_storage_records(t, int(keep), stream or None))


SPT_L2_BLOCK_ROWS_DEFAULT = 196608


def build_mode_l2_blocks(t: int, mode: int, blocked_mode: int = -1, block_rows: int = -1, stream: int = 0):
    _chk(_L.build_mode_l2_blocks(t, mode, blocked_mode, block_rows, stream or None))


def tensor_l2_blocks(t: int, mode: int):
    """(blocked mode or -1, rows per block, groups) of the mode's L2-blocked copy."""
    bm, rows, groups = C.c_int(), C.c_int64(), C.c_int64()
    _chk(_L.tensor_l2_blocks(t, mode, C.byref(bm), C.byref(rows), C.byref(groups)))
    return bm.value, rows.value, groups.value


def tensor_create_shard(t: int, mode: int, begin: int, end: int, stream: int = 0) -> int:
    """Handle of a new tensor holding perm_n positions [begin, end) of t."""
    out = _vp()
    _chk(_L.tensor_create_shard(t, mode, int(begin), int(end), stream or None, C.byref(out)))
    return out.value


def cp_als_hinv(G_ptr: int, order: int, mode: int, rank: int, hinv_ptr: int, status_ptr: int, stream: int = 0):
    _chk(_L.cp_als_hinv(G_ptr, order, mode, rank, hinv_ptr, status_ptr, stream or None))


def cp_als_apply(V_ptr: int, rows: int, ld: int, rank: int, hinv_ptr: int, A32_ptr: int, colsq_ptr: int,
                 stream: int = 0):
    _chk(_L.cp_als_apply(V_ptr or None, int(rows), ld, rank, hinv_ptr, A32_ptr or None, colsq_ptr, stream or None))


def cp_als_normalize(A32_ptr: int, V_ptr: Optional[int], rows: int, ld: int, rank: int, colsq_ptr: int, A_ptr: int,
                     fdt, lambda_ptr: int, inner_ptr: Optional[int], stream: int = 0):
    _chk(_L.cp_als_normalize(A32_ptr or None, V_ptr or None, int(rows), ld, rank, colsq_ptr, A_ptr or None,
                             _dt(fdt), lambda_ptr, inner_ptr or None, stream or None))


def cp_als_gram(A_ptr: int, rows: int, ld: int, rank: int, fdt, G_ptr: int, stream: int = 0):
    _chk(_L.cp_als_gram(A_ptr or None, int(rows), ld, rank, _dt(fdt), G_ptr, stream or None))


def cp_als_fit(G_ptr: int, order: int, rank: int, lambda_ptr: int, inner_ptr: int, xnorm2: float, fit_ptr: int,
               stream: int = 0):
    _chk(_L.cp_als_fit(G_ptr, order, rank, lambda_ptr, inner_ptr, float(xnorm2), fit_ptr, stream or None))


def spt_row_gather_probe(method: int, F1_ptr: int, I1: int, F2_ptr: int, I2: int, r1_ptr: int, r2_ptr: int,
                         n: int, sink_ptr: int, status_ptr: int, stream: int = 0):
    """Enqueue the factor-row gather probe (method 0 loads, 1 TMA gather4, 2 bulk copies)."""
    _chk(_L.spt_row_gather_probe(method, F1_ptr, I1, F2_ptr, I2, r1_ptr, r2_ptr, n, sink_ptr, status_ptr,
                                 stream or None))


def spt_set_wait_tries(tries: int):
    """Try budget of the kernels' bounded waits for later launches (-1 = default)."""
    _chk(_L.spt_set_wait_tries(int(tries)))


def mode_permutation_noalloc(keys_ptr: int, n: int, dim: int, perm_ptr: int, stream: int = 0):
    """Mode permutation computed in the library's static scratch area, for
    callers that cannot allocate device memory (see include/spt.h)."""
    _chk(_L.mode_permutation_noalloc(keys_ptr or None, n, dim, perm_ptr or None, stream or None))


def gcp_gradient(t: int, mode: int, factor_ptrs, fdt, rank: int, ld: int, loss, grad_ptr: int,
                 loss_ptr: int = 0, stream: int = 0):
    arr = (_vp * len(factor_ptrs))(*factor_ptrs)
    lo = LOSSES[loss] if isinstance(loss, str) else int(loss)
    _chk(_L.gcp_gradient(t, mode, arr, _dt(fdt), rank, ld, lo, grad_ptr, loss_ptr or None,
                         stream or None))


def mttkrp_batch_create(items, fdt):
    """items: list of dicts with tensor (handle), mode, rank, ld, factors
    (list of device pointers), outs (list of device pointers), scheds (list of
    spt_schedule or None).  Returns (batch handle, keep-alive list)."""
    arr = (spt_batch_item * len(items))()
    keep = []
    for q, it in enumerate(items):
        f = _ptrs(it["factors"])
        o = _ptrs(it["outs"])
        keep += [f, o]
        sc = None
        if it.get("scheds") is not None:
            sc = (spt_schedule * len(it["scheds"]))(*it["scheds"])
            keep.append(sc)
        arr[q] = spt_batch_item(it["tensor"], it.get("mode", -1), it["rank"], it["ld"], f, o,
                                C.cast(sc, C.POINTER(spt_schedule)) if sc is not None else None)
    keep.append(arr)
    out = _vp()
    _chk(_L.mttkrp_batch_create(len(items), arr, _dt(fdt), C.byref(out)))
    return out.value, keep


def mttkrp_batch_run(b: int, stream: int = 0):
    _chk(_L.mttkrp_batch_run(b, stream or None))


def mttkrp_batch_info(b: int):
    t, i, k = C.c_int64(), C.c_int64(), C.c_int()
    _chk(_L.mttkrp_batch_info(b, C.byref(t), C.byref(i), C.byref(k)))
    return t.value, i.value, k.value


def mttkrp_batch_check(b: int, stream: int = 0):
    _chk(_L.mttkrp_batch_check(b, stream or None))


def mttkrp_batch_destroy(b: int):
    _chk(_L.mttkrp_batch_destroy(b))


def mttkrp_candidates(t: int, mode: int, rank: int):
    """Returns (list of spt_schedule, list of 0/1 valid flags)."""
    out = (spt_schedule * SPT_NUM_CANDIDATES)()
    valid = (C.c_int * SPT_NUM_CANDIDATES)()
    _chk(_L.mttkrp_candidates(t, mode, rank, out, valid))
    return list(out), list(valid)


def mttkrp_time_schedule(t, mode, factor_ptrs, fdt, rank, ld, out_ptr, sched, reps=3, stream=0):
    ms = C.c_float()
    _chk(_L.mttkrp_time_schedule(t, mode, _ptrs(factor_ptrs), _dt(fdt), rank, ld, out_ptr,
                                 C.byref(sched), reps, C.byref(ms), stream or None))
    return ms.value


def mttkrp_autotune(t, mode, factor_ptrs, fdt, rank, ld, out_ptr, reps=2, stream=0):
    """Returns (best spt_schedule, best ms, list of per-candidate ms; -1 invalid)."""
    best = spt_schedule()
    bms = C.c_float()
    times = (C.c_float * SPT_NUM_CANDIDATES)()
    _chk(_L.mttkrp_autotune(t, mode, _ptrs(factor_ptrs), _dt(fdt), rank, ld, out_ptr, reps,
                            C.byref(best), C.byref(bms), times, stream or None))
    return best, bms.value, list(times)


def tensor_mode_features(t, mode, rank, fdt):
    f = (C.c_float * SPT_NUM_FEATURES)()
    _chk(_L.tensor_mode_features(t, mode, rank, _dt(fdt), f))
    return list(f)


def mlp_param_count(F, H1, H2, K):
    return int(_L.mlp_param_count(F, H1, H2, K))


def mlp_workspace_floats(B, F, H1, H2, K):
    return int(_L.mlp_workspace_floats(B, F, H1, H2, K))


def mlp_forward(B, F, H1, H2, K, X_ptr, params_ptr, Y_ptr, work_ptr, stream=0):
    _chk(_L.mlp_forward(B, F, H1, H2, K, X_ptr, params_ptr, Y_ptr, work_ptr, stream or None))


def mlp_loss_grad(B, F, H1, H2, K, X_ptr, params_ptr, T_ptr, M_ptr, grads_ptr, loss_ptr, work_ptr,
                  stream=0):
    _chk(_L.mlp_loss_grad(B, F, H1, H2, K, X_ptr, params_ptr, T_ptr, M_ptr, grads_ptr, loss_ptr,
                          work_ptr, stream or None))


def mlp_adam(n, params_ptr, grads_ptr, m_ptr, v_ptr, lr, beta1, beta2, eps, step, stream=0):
    _chk(_L.mlp_adam(n, params_ptr, grads_ptr, m_ptr, v_ptr, lr, beta1, beta2, eps, step,
                     stream or None))


def mlp_infer(B, F, H1, H2, K, X_ptr, params_ptr, Y_ptr, stream=0):
    _chk(_L.mlp_infer(B, F, H1, H2, K, X_ptr, params_ptr, Y_ptr, stream or None))


def mttkrp_select(t, mode, fdt, rank, sel: "spt_selector", stream=0):
    out = spt_schedule()
    pred = (C.c_float * SPT_NUM_CANDIDATES)()
    _chk(_L.mttkrp_select(t, mode, _dt(fdt), rank, C.byref(sel), C.byref(out), pred, stream or None))
    return out, list(pred)

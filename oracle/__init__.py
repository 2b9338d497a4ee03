"""FP64 CPU oracle for the sparse MTTKRP / CP-ALS path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package's
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline leg, never by
the product library.  The arithmetic lives in ``oracle.c`` (plain C, double
precision, single thread); this wrapper only converts numpy arrays.

Every function takes inputs already widened to float64 where it matters
(``as_f64`` widens fp32 / bf16-bit / f16-bit arrays exactly).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_mttkrp.argtypes = [C.c_int, _lp, C.c_int64, _ip, _dp, C.c_int, C.c_int,
                                    C.POINTER(_dp), _lp, _dp, _dp, C.c_int64]
        L.oracle_mttkrp_threads.argtypes = [C.c_int, _lp, C.c_int64, _ip, _dp, C.c_int, C.c_int,
                                            C.POINTER(_dp), _lp, _dp, _dp, C.c_int64, C.c_int]
        L.oracle_mttkrp_threads.restype = C.c_int
        L.oracle_mttkrp_rows.argtypes = [C.c_int, _lp, C.c_int64, _ip, _dp, C.c_int, C.c_int,
                                         C.POINTER(_dp), _lp, _dp, C.c_int64, _ip, _dp, C.c_int64]
        L.oracle_stable_argsort.argtypes = [C.c_int64, _ip, _ip]
        L.oracle_coalesce.argtypes = [C.c_int, C.c_int64, _ip, _dp, _ip, _dp]
        L.oracle_coalesce.restype = C.c_int64
        L.oracle_norm2.argtypes = [C.c_int, C.c_int64, _ip, _dp]
        L.oracle_norm2.restype = C.c_double
        L.oracle_gram.argtypes = [C.c_int64, C.c_int, _dp, C.c_int64, _dp]
        L.oracle_cholesky.argtypes = [C.c_int, _dp, _dp]
        L.oracle_cholesky.restype = C.c_int
        L.oracle_cp_als_iter.argtypes = [C.c_int, _lp, C.c_int64, _ip, _dp, C.c_int,
                                         C.POINTER(_dp), _dp, C.c_int, C.c_double, _dp]
        L.oracle_cp_als_iter.restype = C.c_int
        L.oracle_round_bf16.argtypes = [C.c_int64, _dp, _dp]
        L.oracle_gcp_grad.argtypes = [C.c_int, _lp, C.c_int64, _ip, _dp, C.c_int, C.c_int,
                                      C.POINTER(_dp), _lp, C.c_int, _dp, C.c_int64]
        L.oracle_gcp_grad.restype = C.c_double
        L.oracle_mlp_forward.argtypes = [C.c_int] * 5 + [_dp] * 10
        L.oracle_mlp_loss_grad.argtypes = [C.c_int] * 5 + [_dp] * 15
        L.oracle_mlp_loss_grad.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _l(a):
    return a.ctypes.data_as(_lp)


def as_f64(a, dtype: str = "f32") -> np.ndarray:
    """Exact widening to float64 of fp32 data or of bf16 / f16 bit patterns."""
    a = np.asarray(a)
    if dtype == "bf16":
        a = (a.astype(np.uint16).astype(np.uint32) << 16).view(np.float32)
    elif dtype == "f16":
        a = a.astype(np.uint16).view(np.float16)
    return np.ascontiguousarray(a, dtype=np.float64)


def _prep(idx, vals):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    assert idx.ndim == 2 and idx.shape[1] == vals.shape[0]
    return idx, vals


def _fac_ptrs(factors: Sequence[np.ndarray]):
    fs = [np.ascontiguousarray(f, dtype=np.float64) for f in factors]
    arr = (_dp * len(fs))(*[_d(f) for f in fs])
    lda = np.array([f.shape[1] for f in fs], dtype=np.int64)
    return fs, arr, lda


def mttkrp(idx, vals, dims, factors, n: int, R: int, lam=None, ld: Optional[int] = None):
    """Mode-``n`` MTTKRP by the definition (Sec. 3 eq. mttkrp); returns I_n x ld."""
    idx, vals = _prep(idx, vals)
    d, P = idx.shape
    dims_a = np.array(dims, dtype=np.int64)
    fs, arr, lda = _fac_ptrs(factors)
    ld = R if ld is None else ld
    V = np.zeros((int(dims[n]), ld), dtype=np.float64)
    lam_a = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
    lib().oracle_mttkrp(d, _l(dims_a), P, _i(idx), _d(vals), n, R, arr, _l(lda),
                        None if lam_a is None else _d(lam_a), _d(V), ld)
    return V


def mttkrp_threads(idx, vals, dims, factors, n: int, R: int, threads: int, lam=None,
                   ld: Optional[int] = None):
    """The MTTKRP definition on ``threads`` host threads (the CPU baseline's
    all-core form).  Thread t owns a contiguous range of output rows, cut so
    that each range holds about P/threads nonzeros; every thread walks all
    nonzeros in storage order and applies only those of its own rows, so each
    row receives its additions in the serial order and the result is
    bit-identical to ``mttkrp`` for any thread count."""
    idx, vals = _prep(idx, vals)
    d, P = idx.shape
    dims_a = np.array(dims, dtype=np.int64)
    fs, arr, lda = _fac_ptrs(factors)
    ld = R if ld is None else ld
    V = np.zeros((int(dims[n]), ld), dtype=np.float64)
    lam_a = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
    if lib().oracle_mttkrp_threads(d, _l(dims_a), P, _i(idx), _d(vals), n, R, arr, _l(lda),
                                   None if lam_a is None else _d(lam_a), _d(V), ld, int(threads)):
        raise MemoryError("oracle_mttkrp_threads: thread or array creation failed")
    return V


def mttkrp_rows(idx, vals, dims, factors, n: int, R: int, rows, lam=None):
    """Selected rows of the mode-``n`` MTTKRP (same definition); nrows x R."""
    idx, vals = _prep(idx, vals)
    d, P = idx.shape
    dims_a = np.array(dims, dtype=np.int64)
    fs, arr, lda = _fac_ptrs(factors)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    V = np.zeros((rows.shape[0], R), dtype=np.float64)
    lam_a = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
    lib().oracle_mttkrp_rows(d, _l(dims_a), P, _i(idx), _d(vals), n, R, arr, _l(lda),
                             None if lam_a is None else _d(lam_a), rows.shape[0], _i(rows),
                             _d(V), R)
    return V


GCP_LOSSES = {"poisson": 0, "bernoulli": 1, "gaussian": 2}


def gcp_grad(idx, vals, dims, factors, n: int, R: int, loss: str, ld: Optional[int] = None):
    """Generalised CP loss F and its gradient with respect to A^(n) (I_n x ld),
    by the definition in ``oracle.c`` (Poisson over every entry of the
    tensor, Bernoulli-logit and Gaussian over the stored entries)."""
    idx, vals = _prep(idx, vals)
    d, P = idx.shape
    dims_a = np.array(dims, dtype=np.int64)
    fs, arr, lda = _fac_ptrs(factors)
    ld = R if ld is None else ld
    G = np.zeros((int(dims[n]), ld), dtype=np.float64)
    F = lib().oracle_gcp_grad(d, _l(dims_a), P, _i(idx), _d(vals), n, R, arr, _l(lda),
                              GCP_LOSSES[loss], _d(G), ld)
    return G, F


def stable_argsort(keys) -> np.ndarray:
    """Positions ordered by (key, position) -- the mode permutation of Sec. 6."""
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    perm = np.empty(keys.shape[0], dtype=np.int32)
    lib().oracle_stable_argsort(keys.shape[0], _i(keys), _i(perm))
    return perm


def coalesce(idx, vals):
    """Distinct coordinates in lexicographic order and their FP64 value sums."""
    idx, vals = _prep(idx, vals)
    d, P = idx.shape
    oi = np.zeros((d, max(P, 1)), dtype=np.int32)
    ov = np.zeros(max(P, 1), dtype=np.float64)
    u = lib().oracle_coalesce(d, P, _i(idx), _d(vals), _i(oi), _d(ov))
    return np.ascontiguousarray(oi[:, :u]), ov[:u].copy()


def norm2(idx, vals) -> float:
    idx, vals = _prep(idx, vals)
    return float(lib().oracle_norm2(idx.shape[0], idx.shape[1], _i(idx), _d(vals)))


def gram(A, R: Optional[int] = None):
    A = np.ascontiguousarray(A, dtype=np.float64)
    R = A.shape[1] if R is None else R
    G = np.zeros((R, R))
    lib().oracle_gram(A.shape[0], R, _d(A), A.shape[1], _d(G))
    return G


def cholesky(H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    L = np.zeros_like(H)
    st = lib().oracle_cholesky(H.shape[0], _d(H), _d(L))
    return L if st == 0 else None


def cp_als_iter(idx, vals, dims, factors: List[np.ndarray], R: int, bf16: bool = False,
                xnorm2: Optional[float] = None):
    """One CP-ALS iteration over all modes.  ``factors`` are I_m x R float64
    (updated in place).  Returns ``(lambda, fit, status)``."""
    idx, vals = _prep(idx, vals)
    d, P = idx.shape
    for f in factors:
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape[1] == R
    dims_a = np.array(dims, dtype=np.int64)
    arr = (_dp * d)(*[_d(f) for f in factors])
    lam = np.zeros(R)
    fit = np.zeros(1)
    x2 = norm2(idx, vals) if xnorm2 is None else xnorm2
    st = lib().oracle_cp_als_iter(d, _l(dims_a), P, _i(idx), _d(vals), R, arr, _d(lam),
                                  int(bf16), x2, _d(fit))
    return lam, float(fit[0]), int(st)


def round_bf16(x) -> np.ndarray:
    """Each float64 value rounded to the nearest bfloat16 value (ties to
    even, bfloat16 subnormals, overflow to infinity); returned as float64.
    The rounding the bf16 CP-ALS oracle applies to updated factors."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().oracle_round_bf16(x.size, _d(x), _d(y))
    return y


def mlp_forward(X, params):
    W1, b1, W2, b2, W3, b3 = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    X = np.ascontiguousarray(X, dtype=np.float64)
    B, F = X.shape
    H1, H2, K = W1.shape[0], W2.shape[0], W3.shape[0]
    h1 = np.zeros((B, H1)); h2 = np.zeros((B, H2)); Y = np.zeros((B, K))
    lib().oracle_mlp_forward(B, F, H1, H2, K, _d(X), _d(W1), _d(b1), _d(W2), _d(b2),
                             _d(W3), _d(b3), _d(h1), _d(h2), _d(Y))
    return Y


def mlp_loss_grad(X, params, T, M):
    W1, b1, W2, b2, W3, b3 = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    B, F = X.shape
    H1, H2, K = W1.shape[0], W2.shape[0], W3.shape[0]
    grads = [np.zeros_like(p) for p in (W1, b1, W2, b2, W3, b3)]
    loss = lib().oracle_mlp_loss_grad(B, F, H1, H2, K, _d(X), _d(W1), _d(b1), _d(W2),
                                      _d(b2), _d(W3), _d(b3), _d(T), _d(M),
                                      *[_d(g) for g in grads])
    return float(loss), grads

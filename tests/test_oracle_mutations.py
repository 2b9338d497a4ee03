"""The MTTKRP pins catch plausible mistakes planted in a copy of the oracle.

Each case compiles ``oracle.c`` with one deliberate defect (a dropped term,
a wrong index, a sum instead of a product, an overwrite instead of an
accumulation) into a temporary library and checks that the dense-unfolding
pin rejects it.  The defects live only in the temporary copy.
"""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

import synth
from tests.test_oracle_pins import _bf16_pin_values, _dense, _khatri_rao_unfold_mttkrp, _ref_bf16

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTATIONS = {
    "own_factor_included": ("            if (m == n) continue;\n                int64_t row",
                            "            (void)0;\n                int64_t row"),
    "output_row_from_mode0": ("int64_t k = idx[(int64_t)n * P + i];\n        for (int j = 0; j < R; ++j) {\n            double t = vals[i];\n            for (int m = 0; m < d; ++m) {\n                if (m == n) continue;\n                int64_t row",
                              "int64_t k = idx[(int64_t)0 * P + i] % In;\n        for (int j = 0; j < R; ++j) {\n            double t = vals[i];\n            for (int m = 0; m < d; ++m) {\n                if (m == n) continue;\n                int64_t row"),
    "sum_not_product": ("t *= A[m][row * lda[m] + j];", "t += A[m][row * lda[m] + j];"),
    "transposed_factor": ("t *= A[m][row * lda[m] + j];", "t *= A[m][(j % dims[m]) * lda[m] + (row % R)];"),
    "overwrite_not_accumulate": ("V[k * ldv + j] += t;\n        }\n    }\n    if (lambda)\n        for (int64_t k = 0; k < In; ++k)",
                                 "V[k * ldv + j] = t;\n        }\n    }\n    if (lambda)\n        for (int64_t k = 0; k < In; ++k)"),
    "lambda_dropped": ("for (int j = 0; j < R; ++j) V[k * ldv + j] *= lambda[j];",
                       "for (int j = 0; j < R; ++j) V[k * ldv + j] *= 1.0;"),
}


def _build_variant(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    cpath = os.path.join(tmp, f"{name}.c")
    open(cpath, "w").write(src)
    so = os.path.join(tmp, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", cpath, "-o", so, "-lm"])
    return C.CDLL(so)


def _run(L, idx, vals, dims, facs, n, R, lam):
    dp = C.POINTER(C.c_double)
    fs = [np.ascontiguousarray(f, dtype=np.float64) for f in facs]
    arr = (dp * len(fs))(*[f.ctypes.data_as(dp) for f in fs])
    lda = np.array([f.shape[1] for f in fs], dtype=np.int64)
    dims_a = np.array(dims, dtype=np.int64)
    V = np.zeros((dims[n], R))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    v64 = np.ascontiguousarray(vals, dtype=np.float64)
    L.oracle_mttkrp.argtypes = [C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                                C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    L.oracle_mttkrp(len(dims), dims_a.ctypes.data, idx.shape[1], idx.ctypes.data, v64.ctypes.data,
                    n, R, C.cast(arr, C.c_void_p), lda.ctypes.data, lam.ctypes.data, V.ctypes.data, R)
    return V


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_dense_pin_rejects_planted_mistake(name):
    dims = (7, 6, 5)
    R = 4
    idx, vals = synth.coo_uniform(dims, 80, 31)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 31, "normal")]
    lam = np.array([0.5, 1.5, 2.0, 0.75])
    X = _dense(idx, vals, dims)
    with tempfile.TemporaryDirectory() as tmp:
        L = _build_variant(name, *MUTATIONS[name], tmp)
        caught = False
        for n in range(3):
            ref = _khatri_rao_unfold_mttkrp(X, facs, n, R) * lam[None, :]
            got = _run(L, idx, vals, dims, facs, n, R, lam)
            if not np.allclose(got, ref, rtol=1e-12, atol=1e-12):
                caught = True
        assert caught, f"planted mistake {name} passed the dense pin"


# planted mistakes in the generalised CP gradient, caught by the dense-loss /
# finite-difference pin of tests/test_oracle_pins.py
GCP_MUTATIONS = {
    "poisson_sign": ("            y = -x / m;                 /* the stored entry's part of 1 - x/m */",
                     "            y = x / m;"),
    "dense_term_dropped": ("            for (int64_t k = 0; k < In; ++k) G[k * ldg + j] += c;",
                           "            (void)c;"),
    "own_mode_in_dense_term": ("                if (l != n) c *= cs;", "                c *= cs;"),
    "bernoulli_derivative": ("            y = 1.0 / (1.0 + exp(-m)) - x;", "            y = 1.0 / (1.0 + exp(m)) - x;"),
    "gaussian_factor_two": ("            y = 2.0 * (m - x);", "            y = (m - x);"),
    "own_factor_in_product": ("            for (int l = 0; l < d; ++l) {\n                if (l == n) continue;\n                t *= A[l]",
                              "            for (int l = 0; l < d; ++l) {\n                t *= A[l]"),
}


@pytest.mark.parametrize("name", sorted(GCP_MUTATIONS))
def test_gcp_pin_rejects_planted_mistake(name):
    from tests.test_oracle_pins import _gcp_loss_dense
    dims = (5, 4, 3)
    R = 2
    idx, vals = synth.coo_zipf(dims, 30, 0.7, 9)
    rng = np.random.default_rng(2)
    A = [rng.random((I, R)) + 0.2 for I in dims]
    dp = C.POINTER(C.c_double)
    fs = [np.ascontiguousarray(a) for a in A]
    arr = (dp * 3)(*[f.ctypes.data_as(dp) for f in fs])
    lda = np.array([R] * 3, dtype=np.int64)
    dims_a = np.array(dims, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    caught = False
    with tempfile.TemporaryDirectory() as tmp:
        L = _build_variant(name, *GCP_MUTATIONS[name], tmp)
        L.oracle_gcp_grad.argtypes = [C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                                      C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int64]
        L.oracle_gcp_grad.restype = C.c_double
        for loss, code in (("poisson", 0), ("bernoulli", 1), ("gaussian", 2)):
            v = vals if loss != "bernoulli" else (vals > 0.5).astype(np.float32)
            v64 = np.ascontiguousarray(v, dtype=np.float64)
            for n in range(3):
                G = np.zeros((dims[n], R))
                F = L.oracle_gcp_grad(3, dims_a.ctypes.data, idx.shape[1], idx.ctypes.data, v64.ctypes.data,
                                      n, R, C.cast(arr, C.c_void_p), lda.ctypes.data, code, G.ctypes.data, R)
                Fd = _gcp_loss_dense(idx, v, dims, A, loss)
                h = 1e-6
                fd = np.zeros_like(G)
                for k in range(dims[n]):
                    for j in range(R):
                        Ap = [a.copy() for a in A]
                        Am = [a.copy() for a in A]
                        Ap[n][k, j] += h
                        Am[n][k, j] -= h
                        fd[k, j] = (_gcp_loss_dense(idx, v, dims, Ap, loss) -
                                    _gcp_loss_dense(idx, v, dims, Am, loss)) / (2 * h)
                if abs(F - Fd) > 1e-10 * max(1.0, abs(Fd)) or np.abs(G - fd).max() > 1e-6 * max(1.0, np.abs(fd).max()):
                    caught = True
    assert caught, f"planted mistake {name} passed the generalised CP pin"


# planted mistakes in the all-core form, caught by its pins (dense unfolding,
# bit-identical to the serial definition)
THREAD_MUTATIONS = {
    "boundary_row_twice": ("if (k < w->lo || k >= w->hi) continue;", "if (k < w->lo || k > w->hi) continue;"),
    "overwrite_not_accumulate": ("w->V[k * w->ldv + j] += t;", "w->V[k * w->ldv + j] = t;"),
    "last_row_dropped": ("w->hi = (t + 1 < T) ? jobs[t + 1].lo : In;", "w->hi = (t + 1 < T) ? jobs[t + 1].lo : In - 1;"),
    "lambda_twice": ("        for (int64_t k = w->lo; k < w->hi; ++k)\n            for (int j = 0; j < w->R; ++j) w->V[k * w->ldv + j] *= w->lambda[j];",
                     "        for (int64_t k = w->lo; k < w->hi; ++k)\n            for (int j = 0; j < w->R; ++j) w->V[k * w->ldv + j] *= w->lambda[j] * w->lambda[j];"),
}


@pytest.mark.parametrize("name", sorted(THREAD_MUTATIONS))
def test_thread_pins_reject_planted_mistake(name):
    dims = (9, 7, 5)
    R = 4
    idx, vals = synth.coo_uniform(dims, 150, 33)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 33, "normal")]
    lam = np.array([0.5, 1.5, 2.0, 0.75])
    X = _dense(idx, vals, dims)
    dp = C.POINTER(C.c_double)
    fs = [np.ascontiguousarray(f) for f in facs]
    arr = (dp * 3)(*[f.ctypes.data_as(dp) for f in fs])
    lda = np.array([R] * 3, dtype=np.int64)
    dims_a = np.array(dims, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    v64 = np.ascontiguousarray(vals, dtype=np.float64)
    caught = False
    with tempfile.TemporaryDirectory() as tmp:
        L = _build_variant(name, *THREAD_MUTATIONS[name], tmp)
        L.oracle_mttkrp_threads.argtypes = [C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                                            C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                            C.c_int]
        for T in (3, 8):
            for n in range(3):
                V = np.zeros((dims[n], R))
                L.oracle_mttkrp_threads(3, dims_a.ctypes.data, idx.shape[1], idx.ctypes.data, v64.ctypes.data, n,
                                        R, C.cast(arr, C.c_void_p), lda.ctypes.data, lam.ctypes.data,
                                        V.ctypes.data, R, T)
                ref = _khatri_rao_unfold_mttkrp(X, facs, n, R) * lam[None, :]
                if not np.allclose(V, ref, rtol=1e-12, atol=1e-12):
                    caught = True
    assert caught, f"planted mistake {name} passed the all-core pins"


# Plausible mistakes in the oracle's bf16 rounding (the step the bf16 CP-ALS
# oracle applies to each updated factor); the bit-level pin must reject each.
ROUND_MUTATIONS = {
    "truncation": ("double q = nearbyint(ldexp(m, bits));", "double q = trunc(ldexp(m, bits));"),
    "ties_away_from_zero": ("double q = nearbyint(ldexp(m, bits));", "double q = round(ldexp(m, bits));"),
    "no_subnormal_range": ("int bits = e - 1 >= -126 ? 8 : e + 133;", "int bits = 8;"),
    "no_overflow": ("if (fabs(r) > ldexp(255.0, 120)) return copysign(INFINITY, x);", ""),
    "seven_bits": ("int bits = e - 1 >= -126 ? 8 : e + 133;", "int bits = e - 1 >= -126 ? 7 : e + 132;"),
}


@pytest.mark.parametrize("name", sorted(ROUND_MUTATIONS))
def test_bf16_pin_rejects_planted_rounding_mistake(name):
    x = _bf16_pin_values()
    ref = np.array([_ref_bf16(float(t)) for t in x])
    with tempfile.TemporaryDirectory() as tmp:
        L = _build_variant("round_" + name, *ROUND_MUTATIONS[name], tmp)
        L.oracle_round_bf16.argtypes = [C.c_int64, C.c_void_p, C.c_void_p]
        y = np.empty_like(x)
        L.oracle_round_bf16(x.size, x.ctypes.data, y.ctypes.data)
    assert (y.view(np.uint64) != ref.view(np.uint64)).any(), f"planted mistake {name} passed the bf16 pin"

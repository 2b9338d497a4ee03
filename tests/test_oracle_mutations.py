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
from tests.test_oracle_pins import _dense, _khatri_rao_unfold_mttkrp

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

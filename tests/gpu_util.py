"""Helpers for the GPU parity tests: move synthetic inputs to the device and
compare the CUDA path's results with the oracle's."""
import numpy as np
import torch

import oracle
import synth

TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "f64": torch.float64}


def to_device_factor(f, dtype):
    """synth factor (float32 / float64 array or uint16 bit pattern) -> CUDA tensor."""
    if dtype in ("f32", "f64"):
        return torch.from_numpy(np.ascontiguousarray(f)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(f).view(np.int16)).cuda()
    return t.view(TORCH_DT[dtype])


def widen(f, dtype, R):
    """Exact float64 view of a synth factor's first R columns."""
    return oracle.as_f64(f, dtype)[:, :R].copy()


def rel_fro(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


# Tolerances (relative Frobenius error vs the FP64 oracle fed the same stored
# factor values).  fp32 accumulation of products of exactly representable
# inputs: ~ sqrt(terms per row) * 2^-24 per element; 1e-5 is the stated bound.
TOL = {"f32": 1e-5, "bf16": 2e-3, "f16": 2e-3, "f64": 1e-12}


def elementwise_bound(got, ref, scale):
    """Every element within 1e-5 of the row's magnitude scale (sum of |terms|)."""
    err = np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))
    return float((err / np.maximum(scale, 1e-30)).max())

"""Seeded synthetic inputs for the sparse MTTKRP / CP-ALS path.

This module only *draws* inputs: COO coordinates, nonzero values and factor
matrices, with the shapes and distributions of the workloads the method is
measured on.  It holds none of the method's arithmetic (no MTTKRP, no Gram,
no solve), so both the CPU oracle and the CUDA path can be fed from it.

Conventions
-----------
* Coordinates are 0-based ``int32`` arrays, mode-major: ``idx[m, i]`` is the
  mode-``m`` coordinate of nonzero ``i`` (the paper's ``l_{i,m+1}``).
* Values are ``float32``.
* Factor matrices are row-major ``I_m x ld`` arrays (``ld >= R``, a multiple
  of 8); columns ``R..ld-1`` are zero.  16-bit factors are returned as their
  bit patterns (``uint16``): ``bf16`` rounded from the fp32 draw with
  round-to-nearest-even by torch's CPU conversion, ``f16`` by numpy's.
* Every draw comes from ``numpy.random.Generator(PCG64)`` streams spawned from
  one ``SeedSequence(seed)``, one stream per purpose, so a component does not
  change when another one is drawn differently.

Power-law ("Zipf") coordinates: rank ``k = 1..I`` is drawn with probability
``k^-s / sum_q q^-s`` by inverse CDF (``s = 0`` is uniform), and rank ``k``
is placed at index ``(a*(k-1) + b) mod I`` with ``gcd(a, I) = 1`` so the hot
rows are scattered over the mode.  Modes are independent.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "workload",
    "coo_zipf", "coo_uniform_distinct", "coo_uniform", "factor_matrices",
    "small_integer_case", "padded_ld", "bf16_bits_to_f32", "f16_bits_to_f32",
    "batched_specs", "selector_specs",
]

_CHUNK = 1 << 24  # draws per inverse-CDF batch (bounds temporary memory)


def padded_ld(R: int) -> int:
    """Row stride (elements) for rank ``R``: ``R`` rounded up to a multiple of 8."""
    return max(8, (R + 7) // 8 * 8)


def _gens(seed: int, n: int) -> List[np.random.Generator]:
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(n)]


def _zipf_indices(rng: np.random.Generator, I: int, count: int, s: float) -> np.ndarray:
    """``count`` independent power-law coordinates in ``[0, I)`` (int32)."""
    out = np.empty(count, dtype=np.int32)
    if I == 1 or count == 0:
        out[:] = 0
        return out
    # affine bijection rank -> index, drawn first so it does not depend on count
    while True:
        a = int(rng.integers(1, I))
        if math.gcd(a, I) == 1:
            break
    b = int(rng.integers(0, I))
    if s == 0.0:
        for c0 in range(0, count, _CHUNK):
            c1 = min(count, c0 + _CHUNK)
            r = rng.integers(0, I, size=c1 - c0, dtype=np.int64)
            out[c0:c1] = ((a * r + b) % I).astype(np.int32)
        return out
    import torch  # CPU searchsorted is multi-threaded; used as a library lookup

    w = np.arange(1, I + 1, dtype=np.float64) ** (-float(s))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf_t = torch.from_numpy(cdf)
    for c0 in range(0, count, _CHUNK):
        c1 = min(count, c0 + _CHUNK)
        u = rng.random(c1 - c0)
        r = torch.searchsorted(cdf_t, torch.from_numpy(u), right=True).numpy()
        np.minimum(r, I - 1, out=r)  # guards u == 1.0 after cdf rounding
        out[c0:c1] = ((a * r + b) % I).astype(np.int32)
    return out


def coo_zipf(dims: Sequence[int], nnz: int, s, seed: int):
    """COO tensor with independent power-law coordinates per mode.

    ``s`` is one exponent or one per mode.  Values are U(0,1) float32.
    Duplicated coordinates are kept (they are additive in the tensor).
    Returns ``(idx[d, nnz] int32, vals[nnz] float32)``.
    """
    d = len(dims)
    ss = [float(s)] * d if np.isscalar(s) else [float(x) for x in s]
    assert len(ss) == d
    g = _gens(seed, d + 1)
    idx = np.empty((d, nnz), dtype=np.int32)
    for m in range(d):
        idx[m] = _zipf_indices(g[m], int(dims[m]), nnz, ss[m])
    vals = g[d].random(nnz, dtype=np.float32)
    return idx, vals


def coo_uniform(dims: Sequence[int], nnz: int, seed: int):
    """COO tensor with independent uniform coordinates (duplicates possible)."""
    return coo_zipf(dims, nnz, 0.0, seed)


def coo_uniform_distinct(dims: Sequence[int], nnz: int, seed: int):
    """COO tensor with ``nnz`` distinct uniformly placed coordinates.

    Positions are drawn without replacement from the dense index space, in
    the random order of the draw (the storage order is not sorted).
    """
    total = int(np.prod([int(x) for x in dims], dtype=np.int64))
    assert nnz <= total
    g = _gens(seed, 2)
    lin = g[0].choice(total, size=nnz, replace=False)
    idx = np.stack(np.unravel_index(lin, tuple(int(x) for x in dims))).astype(np.int32)
    vals = g[1].random(nnz, dtype=np.float32)
    return np.ascontiguousarray(idx), vals


def _to_bf16_bits(x: np.ndarray) -> np.ndarray:
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(
        torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    """Exact widening of bf16 bit patterns to float32."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def f16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    """Exact widening of f16 bit patterns to float32."""
    return np.asarray(b, dtype=np.uint16).view(np.float16).astype(np.float32)


def factor_matrices(dims: Sequence[int], R: int, seed: int, dist: str = "uniform",
                    ld: Optional[int] = None, dtype: str = "f32"):
    """One ``I_m x ld`` row-major factor matrix per mode, padding columns zero.

    ``dist``: ``"uniform"`` (U(0,1)) or ``"normal"`` (N(0,1)).
    ``dtype``: ``"f32"`` -> float32 arrays; ``"bf16"`` / ``"f16"`` -> uint16
    bit patterns of the fp32 draw rounded to nearest even; ``"f64"`` ->
    float64 arrays of a float64 draw.
    """
    ld = padded_ld(R) if ld is None else ld
    assert ld >= R
    g = _gens(seed + 1_000_003, len(dims))
    out = []
    for m, I in enumerate(dims):
        if dtype == "f64":
            if dist == "uniform":
                a = g[m].random((int(I), R))
            elif dist == "normal":
                a = g[m].standard_normal((int(I), R))
            elif dist == "int":
                a = g[m].integers(-3, 4, size=(int(I), R)).astype(np.float64)
            else:
                raise ValueError(dist)
            full = np.zeros((int(I), ld))
            full[:, :R] = a
            out.append(full)
            continue
        if dist == "uniform":
            a = g[m].random((int(I), R), dtype=np.float32)
        elif dist == "normal":
            a = g[m].standard_normal((int(I), R), dtype=np.float32)
        elif dist == "int":  # small integers in {-3..3}
            a = g[m].integers(-3, 4, size=(int(I), R)).astype(np.float32)
        else:
            raise ValueError(dist)
        full = np.zeros((int(I), ld), dtype=np.float32)
        full[:, :R] = a
        if dtype == "f32":
            out.append(full)
        elif dtype == "bf16":
            out.append(_to_bf16_bits(full))
        elif dtype == "f16":
            out.append(full.astype(np.float16).view(np.uint16))
        else:
            raise ValueError(dtype)
    return out


def small_integer_case(dims: Sequence[int], nnz: int, R: int, seed: int, dtype="f32"):
    """Integer-valued case: values in {1..4}, factors in {-3..3}.

    Every product and every partial sum is an integer; while the partial sums
    stay below 2^24 every fp32 summation order gives the same exact result,
    and the integers -3..3 are exact in bf16 and f16 too.
    """
    g = _gens(seed, 2)
    d = len(dims)
    idx = np.stack([g[0].integers(0, int(I), size=nnz) for I in dims]).astype(np.int32)
    vals = g[1].integers(1, 5, size=nnz).astype(np.float32)
    facs = factor_matrices(dims, R, seed, dist="int", dtype=dtype)
    return np.ascontiguousarray(idx), vals, facs


@dataclass
class Workload:
    """A named synthetic workload: shape, skew, rank and factor recipe."""
    name: str
    dims: List[int]
    nnz: int
    s: object  # float or per-mode list; None = distinct uniform
    R: int
    factor_dist: str
    seed: int = 0
    factor_dtype: str = "f32"
    extra: dict = field(default_factory=dict)

    def coo(self):
        if self.s is None:
            return coo_uniform_distinct(self.dims, self.nnz, self.seed)
        return coo_zipf(self.dims, self.nnz, self.s, self.seed)

    def factors(self, R: Optional[int] = None, dtype: Optional[str] = None):
        return factor_matrices(self.dims, R or self.R, self.seed, self.factor_dist,
                               dtype=dtype or self.factor_dtype)


WORKLOADS = {
    # 100x80x60, 10k distinct uniform nonzeros, R=16 U(0,1) factors
    "uniform3d_100x80x60_nnz1e4": Workload(
        "uniform3d_100x80x60_nnz1e4", [100, 80, 60], 10_000, None, 16, "uniform", 0),
    # 1e6 x 5e5 x 2e5, 1e8 nonzeros, Zipf(1.2) per mode, R=16 N(0,1)
    "zipf3d_1e6x5e5x2e5_nnz1e8": Workload(
        "zipf3d_1e6x5e5x2e5_nnz1e8", [1_000_000, 500_000, 200_000], 100_000_000,
        1.2, 16, "normal", 0),
    # 2e6 x 1e5 x 1e4 x 1e3, 2e8 nonzeros, Zipf (1.0, 1.2, 0.8, 0.5), R=32/64
    "zipf4d_2e6x1e5x1e4x1e3_nnz2e8": Workload(
        "zipf4d_2e6x1e5x1e4x1e3_nnz2e8", [2_000_000, 100_000, 10_000, 1_000],
        200_000_000, [1.0, 1.2, 0.8, 0.5], 64, "uniform", 0),
    # the paper's own synthetic tensor (Sec. 7): 30K x 40K x 50K, 1e7 nonzeros at
    # uniformly random coordinates, U(0,1) values and factors; R swept 8..256
    "uniform3d_30kx40kx50k_nnz1e7": Workload(
        "uniform3d_30kx40kx50k_nnz1e7", [30_000, 40_000, 50_000], 10_000_000, 0.0, 128,
        "uniform", 0),
    # 5e5 x 2e5 x 5e4 x 5e3 x 5e2, 3e8 nonzeros, Zipf(1.1), R=32 bf16
    "zipf5d_5e5x2e5x5e4x5e3x5e2_nnz3e8": Workload(
        "zipf5d_5e5x2e5x5e4x5e3x5e2_nnz3e8", [500_000, 200_000, 50_000, 5_000, 500],
        300_000_000, 1.1, 32, "uniform", 0, "bf16"),
}


def workload(name: str, scale: float = 1.0) -> Workload:
    """Named workload; ``scale`` < 1 shrinks nnz (and dims by its cube root)."""
    w = WORKLOADS[name]
    if scale == 1.0:
        return w
    f = scale ** (1.0 / 3.0)
    return Workload(w.name + f"@{scale:g}", [max(2, int(x * f)) for x in w.dims],
                    max(1, int(w.nnz * scale)), w.s, w.R, w.factor_dist, w.seed,
                    w.factor_dtype)


def _log_uniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def batched_specs(count: int = 64, seed0: int = 0, nnz_scale: float = 1.0):
    """Recipe of the many-tensor batch: order 3 or 4, dims log-uniform in
    [1e3, 1e6], nnz log-uniform in [1e4, 5e6], Zipf s ~ U(0, 1.5),
    R in {16, 32, 64}; tensor ``t`` uses seed ``seed0 + t``."""
    out = []
    for t in range(count):
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed0 + t, 7])))
        d = int(rng.integers(3, 5))
        dims = [int(round(_log_uniform(rng, 1e3, 1e6))) for _ in range(d)]
        nnz = max(1, int(round(_log_uniform(rng, 1e4, 5e6) * nnz_scale)))
        s = float(rng.uniform(0.0, 1.5))
        R = int(rng.choice([16, 32, 64]))
        out.append(Workload(f"batch{t}", dims, nnz, s, R, "uniform", seed0 + t))
    return out


def selector_specs(count: int = 500, seed0: int = 10_000, nnz_lo: float = 1e5,
                   nnz_hi: float = 3e7, large: int = 0, large_hi: float = 1.5e8):
    """Recipe of the schedule-selector training tensors: order 3..5, Zipf
    s ~ U(0, 2), R in [8, 128], dims log-uniform in [1e2, 1e6], nnz
    log-uniform in [nnz_lo, nnz_hi]; the last ``large`` tensors draw nnz
    log-uniform in [nnz_hi, large_hi] instead."""
    out = []
    for t in range(count):
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed0 + t, 11])))
        d = int(rng.integers(3, 6))
        dims = [int(round(_log_uniform(rng, 1e2, 1e6))) for _ in range(d)]
        lo, hi = (nnz_hi, large_hi) if t >= count - large else (nnz_lo, nnz_hi)
        nnz = int(round(_log_uniform(rng, lo, hi)))
        s = float(rng.uniform(0.0, 2.0))
        R = int(rng.integers(8, 129))
        out.append(Workload(f"sel{t}", dims, nnz, s, R, "uniform", seed0 + t))
    return out


def coo_zipf_device(dims: Sequence[int], nnz: int, s, seed: int, device: str = "cuda"):
    """The power-law COO recipe of :func:`coo_zipf`, drawn on the GPU with
    torch's generator (a different random stream than the numpy one; used
    where no oracle comparison is made, e.g. schedule-timing data).
    Returns CUDA tensors (idx[d, nnz] int32, vals[nnz] float32)."""
    import torch

    d = len(dims)
    ss = [float(s)] * d if np.isscalar(s) else [float(x) for x in s]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    idx = torch.empty((d, nnz), dtype=torch.int32, device=device)
    for m in range(d):
        I = int(dims[m])
        if I == 1:
            idx[m].zero_()
            continue
        while True:
            a = int(torch.randint(1, I, (1,), generator=g, device=device).item())
            if math.gcd(a, I) == 1:
                break
        b = int(torch.randint(0, I, (1,), generator=g, device=device).item())
        if ss[m] == 0.0:
            r = torch.randint(0, I, (nnz,), generator=g, device=device, dtype=torch.int64)
        else:
            w = torch.arange(1, I + 1, dtype=torch.float64, device=device) ** (-ss[m])
            cdf = torch.cumsum(w, 0)
            cdf /= cdf[-1].clone()
            u = torch.rand(nnz, generator=g, device=device, dtype=torch.float64)
            r = torch.clamp(torch.searchsorted(cdf, u, right=True), max=I - 1)
        idx[m] = ((a * r + b) % I).to(torch.int32)
    vals = torch.rand(nnz, generator=g, device=device, dtype=torch.float32)
    return idx, vals

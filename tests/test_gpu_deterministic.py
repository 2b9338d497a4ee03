"""GPU: the deterministic MTTKRP (mttkrp_deterministic).  Repeated calls give
bit-identical output; the values match the FP64 oracle within the bounds of
the other traversals; integer-valued cases are exact.  Cases are chosen so
that the per-warp boundary slots are exercised in every arrangement: rows
spanning many warps' ranges (one hot row holding every nonzero, so every
warp's range is that one row), ranges of one chunk, ragged last chunks, lane
groups of 1..32 lanes with one and two column chunks, orders 1-5, lambda."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import TOL, rel_fro, to_device_factor, widen

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1809_09175_gb300 as P
    return P


def _bits(t):
    return t.view(torch.int64 if t.dtype == torch.float64 else torch.int32)


def _oracle(idx, vals, dims, facs, dtype, R, n, lam=None):
    A = [widen(f, dtype, R) for f in facs]
    if lam is not None:
        lam = lam.astype(np.float64) if dtype == "f64" else lam.astype(np.float32).astype(np.float64)
    return oracle.mttkrp(idx, vals, dims, A, n, R, lam=lam)


def _check(P, idx, vals, dims, facs, dtype, R, sched_kw=None, lam=None, reps=3):
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    dev = [to_device_factor(f, dtype) for f in facs]
    lam_t = None
    if lam is not None:
        lam_t = torch.from_numpy(lam.astype(np.float64 if dtype == "f64" else np.float32)).cuda()
    for n in range(len(dims)):
        sched = None
        if sched_kw:
            base = P.mttkrp_default_schedule(T.handle, n, dtype, R).as_dict()
            base["scatter"] = P.SCATTERS["sorted"]
            base.update(sched_kw)
            sched = P.spt_schedule.make(**base)
        first = T.mttkrp(n, dev, R, lam=lam_t, sched=sched, deterministic=True)
        for _ in range(reps - 1):
            again = T.mttkrp(n, dev, R, lam=lam_t, sched=sched, deterministic=True)
            assert torch.equal(_bits(first), _bits(again)), (n, "not bit-identical")
        got = first.cpu().numpy()
        assert np.all(got[:, R:] == 0)
        ref = _oracle(idx, vals, dims, facs, dtype, R, n, lam)
        e = rel_fro(got[:, :R], ref)
        assert e <= TOL[dtype], (n, e)
    T.check()
    T.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "f64"])
@pytest.mark.parametrize("order,R", [(1, 4), (2, 8), (3, 16), (4, 20), (5, 7), (3, 100), (3, 200)])
def test_deterministic_matches_oracle_and_repeats(order, R, dtype):
    if order == 1 and dtype != "f32":
        pytest.skip("an order-1 MTTKRP reads no factor: its output is float32 for every dtype")
    P = _lib()
    dims = [700, 500, 300, 40, 9][:order]
    idx, vals = synth.coo_zipf(dims, 120_001, 1.3, 60 + order)
    facs = synth.factor_matrices(dims, R, 3, "uniform", dtype=dtype)
    _check(P, idx, vals, dims, facs, dtype, R)


@pytest.mark.parametrize("sk", [
    {"lanes_per_nnz": 4, "chunks": 1, "nnz_per_group": 9},      # ragged chunks, 8 groups
    {"lanes_per_nnz": 2, "chunks": 2, "nnz_per_group": 3},      # short chunks
    {"lanes_per_nnz": 32, "chunks": 1, "nnz_per_group": 4},     # one group per warp
    {"lanes_per_nnz": 8, "chunks": 2, "warps_per_cta": 4, "nnz_per_group": 33},
])
def test_deterministic_schedules_with_lambda(sk):
    P = _lib()
    dims = (400, 300, 20)
    R = 16
    idx, vals = synth.coo_zipf(dims, 80_003, (1.4, 0.8, 0.0), 21)
    facs = synth.factor_matrices(dims, R, 4, "normal")
    lam = np.linspace(0.5, 2.0, R)
    _check(P, idx, vals, dims, facs, "f32", R, sched_kw=sk, lam=lam)


def test_deterministic_hot_rows():
    """One row holding every nonzero (every warp's range is that row and only
    its last slot is written), then a mode of 3 rows over 300k nonzeros."""
    P = _lib()
    R = 12
    rng = np.random.default_rng(7)
    P_ = 300_000
    for dims, first in [((50, 40, 30), np.full(P_, 7)), ((3, 40, 30), rng.integers(0, 3, P_))]:
        idx = np.stack([first, rng.integers(0, 40, P_), rng.integers(0, 30, P_)]).astype(np.int32)
        vals = rng.random(P_, dtype=np.float32)
        facs = synth.factor_matrices(dims, R, 1, "uniform")
        _check(P, idx, vals, dims, facs, "f32", R)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_deterministic_integer_case_bit_exact(dtype):
    P = _lib()
    dims = (300, 200, 50, 7)
    R = 13
    idx, vals, facs = synth.small_integer_case(dims, 40_000, R, 5, dtype=dtype)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    dev = [to_device_factor(f, dtype) for f in facs]
    for n in range(4):
        got = T.mttkrp(n, dev, R, deterministic=True).cpu().numpy()
        ref = _oracle(idx, vals, dims, facs, dtype, R, n)
        assert np.abs(ref).max() < 2 ** 24
        np.testing.assert_array_equal(got[:, :R], ref.astype(got.dtype))
    T.close()


def test_deterministic_small_and_empty():
    P = _lib()
    R = 8
    for dims, idx in [((5, 4, 3), np.array([[4], [0], [2]], np.int32)),
                      ((1, 1, 6), np.array([[0, 0, 0], [0, 0, 0], [5, 1, 5]], np.int32))]:
        vals = np.arange(1, idx.shape[1] + 1, dtype=np.float32)
        facs = synth.factor_matrices(dims, R, 2, "uniform")
        _check(P, idx, vals, dims, facs, "f32", R)
    T = P.SparseTensor(np.zeros((3, 0), np.int32), np.zeros(0, np.float32), (10, 9, 8))
    T.build_permutation()
    out = torch.full((10, 8), 7.0, device="cuda")
    T.mttkrp(0, [torch.ones((I, 8), device="cuda") for I in (10, 9, 8)], 8, out=out, deterministic=True)
    assert float(out.abs().max()) == 0.0
    T.close()


def test_deterministic_errors():
    P = _lib()
    dims = (30, 20, 10)
    idx, vals = synth.coo_zipf(dims, 500, 0.5, 1)
    T = P.SparseTensor(idx, vals, dims)
    dev = [torch.rand((I, 8), device="cuda") for I in dims]
    with pytest.raises(P.SptError) as ei:  # no mode-sorted copy yet
        T.mttkrp(0, dev, 8, deterministic=True)
    assert ei.value.status == P.SPT_ESTATE
    T.build_permutation()
    base = P.mttkrp_default_schedule(T.handle, 0, "f32", 8).as_dict()
    base["scatter"] = P.SCATTERS["atomic"]
    with pytest.raises(P.SptError) as ei:
        T.mttkrp(0, dev, 8, sched=P.spt_schedule.make(**base), deterministic=True)
    assert ei.value.status == P.SPT_EINVAL
    big = [torch.rand((I, 304), device="cuda") for I in dims]
    with pytest.raises(P.SptError) as ei:
        T.mttkrp(0, big, 300, deterministic=True)
    assert ei.value.status == P.SPT_EUNSUPPORTED
    T.close()

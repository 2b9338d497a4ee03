"""GPU parity: MTTKRP through the C ABI vs the FP64 oracle, element by element.

Covers every scatter strategy (atomic, permuted via perm_n, permuted over
the mode-sorted copy), fp32 / bf16 / f16 factors, orders 1-5, ranks that are
and are not multiples of the 16-byte column chunk, several launch schedules
(so chunk, group and ragged-tail boundaries move), lambda weights and the
degenerate cases (no nonzeros, one nonzero, one hot row, one-long modes).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import TOL, rel_fro, to_device_factor, widen

pytestmark = pytest.mark.gpu

SCATTERS = ["atomic", "perm", "sorted"]


def _lib():
    import paper_1809_09175_gb300 as P
    return P


def _run(P, idx, vals, dims, facs, dtype, R, scatter, sched_kw=None, lam=None, modes=None):
    T = P.SparseTensor(idx, vals, dims)
    if scatter != "atomic":
        T.build_permutation(-1, index_only=(scatter == "perm"))
    dev = [to_device_factor(f, dtype) for f in facs]
    lam_t = None if lam is None else torch.from_numpy(lam.astype(np.float32)).cuda()
    outs = {}
    for n in (range(len(dims)) if modes is None else modes):
        sched = None
        if sched_kw is not None or scatter is not None:
            base = P.mttkrp_default_schedule(T.handle, n, dtype, R).as_dict()
            base["scatter"] = P.SCATTERS[scatter]
            base.update(sched_kw or {})
            sched = P.spt_schedule.make(**base)
        outs[n] = T.mttkrp(n, dev, R, lam=lam_t, sched=sched).cpu().numpy()
    T.check()
    T.close()
    return outs


def _oracle(idx, vals, dims, facs, dtype, R, n, lam=None):
    A = [widen(f, dtype, R) for f in facs]
    return oracle.mttkrp(idx, vals, dims, A, n, R, lam=None if lam is None else lam.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("scatter", SCATTERS)
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_uniform_100x80x60_all_modes(scatter, dtype):
    P = _lib()
    w = synth.WORKLOADS["uniform3d_100x80x60_nnz1e4"]
    idx, vals = w.coo()
    R = w.R
    facs = synth.factor_matrices(w.dims, R, w.seed, "uniform", dtype=dtype)
    outs = _run(P, idx, vals, w.dims, facs, dtype, R, scatter)
    for n in range(3):
        ref = _oracle(idx, vals, w.dims, facs, dtype, R, n)
        got = outs[n]
        assert np.all(got[:, R:] == 0)
        e = rel_fro(got[:, :R], ref)
        assert e <= TOL[dtype], (n, e)
        np.testing.assert_allclose(got[:, :R], ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("scatter", SCATTERS)
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_integer_case_bit_exact(scatter, dtype):
    P = _lib()
    dims = (300, 200, 50, 7)
    R = 13
    idx, vals, facs = synth.small_integer_case(dims, 40_000, R, 5, dtype=dtype)
    outs = _run(P, idx, vals, dims, facs, dtype, R, scatter, {"nnz_per_group": 9})
    for n in range(4):
        ref = _oracle(idx, vals, dims, facs, dtype, R, n)
        assert np.abs(ref).max() < 2 ** 24
        np.testing.assert_array_equal(outs[n][:, :R], ref.astype(np.float32))


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("scatter", SCATTERS)
def test_orders_zipf(order, scatter):
    P = _lib()
    dims = [3000, 1700, 900, 64, 5][:order]
    R = 20
    idx, vals = synth.coo_zipf(dims, 150_001, 1.2, 17 + order)
    facs = synth.factor_matrices(dims, R, 3, "normal")
    lam = np.linspace(0.25, 2.0, R)
    outs = _run(P, idx, vals, dims, facs, "f32", R, scatter, lam=lam)
    for n in range(order):
        ref = _oracle(idx, vals, dims, facs, "f32", R, n, lam=lam)
        e = rel_fro(outs[n][:, :R], ref)
        assert e <= 1e-5, (n, e)


SCHEDS = [
    {"lanes_per_nnz": 1, "chunks": 1, "nnz_per_group": 5, "warps_per_cta": 1},
    {"lanes_per_nnz": 2, "chunks": 2, "nnz_per_group": 30, "warps_per_cta": 3},
    {"lanes_per_nnz": 4, "chunks": 1, "nnz_per_group": 64, "warps_per_cta": 8},
    {"lanes_per_nnz": 8, "chunks": 2, "nnz_per_group": 17, "warps_per_cta": 16},
    {"lanes_per_nnz": 16, "chunks": 1, "nnz_per_group": 128, "warps_per_cta": 4},
    {"lanes_per_nnz": 32, "chunks": 2, "nnz_per_group": 12, "warps_per_cta": 2, "ctas_per_sm": 1},
]


@pytest.mark.parametrize("sk", range(len(SCHEDS)))
@pytest.mark.parametrize("R", [1, 5, 16, 37, 64, 100])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_schedules_and_ranks(sk, R, dtype):
    P = _lib()
    dims = (5000, 800, 300)
    idx, vals = synth.coo_zipf(dims, 60_003, (1.3, 0.7, 0.0), 9)
    facs = synth.factor_matrices(dims, R, 4, "normal", dtype=dtype)
    for scatter in SCATTERS:
        outs = _run(P, idx, vals, dims, facs, dtype, R, scatter, SCHEDS[sk])
        for n in range(3):
            ref = _oracle(idx, vals, dims, facs, dtype, R, n)
            got = outs[n]
            assert np.all(got[:, R:] == 0)
            e = rel_fro(got[:, :R], ref)
            assert e <= 1e-5, (scatter, n, e)


@pytest.mark.parametrize("scatter", SCATTERS)
def test_degenerate_cases(scatter):
    P = _lib()
    R = 8
    # one hot row holding every nonzero (runs span every chunk and warp)
    dims = (50, 40, 30)
    rng = np.random.default_rng(0)
    P_ = 20_000
    idx = np.stack([np.full(P_, 7), rng.integers(0, 40, P_), rng.integers(0, 30, P_)]).astype(np.int32)
    vals = rng.random(P_, dtype=np.float32)
    facs = synth.factor_matrices(dims, R, 1, "uniform")
    outs = _run(P, idx, vals, dims, facs, "f32", R, scatter)
    for n in range(3):
        ref = _oracle(idx, vals, dims, facs, "f32", R, n)
        assert rel_fro(outs[n][:, :R], ref) <= 1e-5
    # a single nonzero; and modes of length one
    for dims, idx in [((5, 4, 3), np.array([[4], [0], [2]], np.int32)),
                      ((1, 1, 6), np.array([[0, 0, 0], [0, 0, 0], [5, 1, 5]], np.int32))]:
        vals = np.arange(1, idx.shape[1] + 1, dtype=np.float32)
        facs = synth.factor_matrices(dims, R, 2, "uniform")
        outs = _run(P, idx, vals, dims, facs, "f32", R, scatter)
        for n in range(3):
            ref = _oracle(idx, vals, dims, facs, "f32", R, n)
            np.testing.assert_allclose(outs[n][:, :R], ref, rtol=1e-6)


def test_empty_tensor_zeroes_output():
    P = _lib()
    dims = (10, 9, 8)
    T = P.SparseTensor(np.zeros((3, 0), np.int32), np.zeros(0, np.float32), dims)
    T.build_permutation()
    facs = [torch.ones((I, 8), device="cuda") for I in dims]
    out = torch.full((10, 8), 7.0, device="cuda")
    T.mttkrp(0, facs, 8, out=out)
    assert float(out.abs().max()) == 0.0
    T.close()


@pytest.mark.parametrize("P_,K", [(1, 3), (1000, 1), (77_777, 1000), (300_001, 2_000_000)])
def test_permutation_matches_stable_argsort(P_, K):
    P = _lib()
    rng = np.random.default_rng(P_)
    dims = (K, 5)
    idx = np.stack([rng.integers(0, K, P_), rng.integers(0, 5, P_)]).astype(np.int32)
    vals = rng.random(P_, dtype=np.float32)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    for n in range(2):
        perm = T.permutation(n).cpu().numpy()
        np.testing.assert_array_equal(perm, oracle.stable_argsort(idx[n]))
    T.close()


def test_coalesce_matches_oracle():
    P = _lib()
    dims = (40, 30, 20, 10)
    idx, vals = synth.coo_zipf(dims, 200_000, 1.4, 12)
    T = P.SparseTensor(idx, vals, dims, coalesce=True)
    ci, cv = oracle.coalesce(idx, vals)
    gi, gv = T.coo()
    np.testing.assert_array_equal(gi.cpu().numpy(), ci)
    np.testing.assert_array_equal(gv.cpu().numpy(), cv.astype(np.float32))
    x2 = float((cv.astype(np.float32).astype(np.float64) ** 2).sum())
    assert abs(T.norm2() - x2) <= 1e-12 * x2
    T.close()


def test_out_of_range_coordinate_is_rejected():
    P = _lib()
    idx = np.array([[0, 1], [0, 5]], np.int32)
    with pytest.raises(P.SptError) as ei:
        P.SparseTensor(idx, np.ones(2, np.float32), (2, 5))
    assert ei.value.status == P.SPT_ERANGE


def test_bad_arguments_return_status():
    P = _lib()
    dims = (10, 9, 8)
    idx, vals = synth.coo_uniform(dims, 100, 1)
    T = P.SparseTensor(idx, vals, dims)
    facs = [torch.ones((I, 8), device="cuda") for I in dims]
    out = torch.empty((10, 8), device="cuda")
    ptrs = [f.data_ptr() for f in facs]
    with pytest.raises(P.SptError) as ei:
        P.mttkrp(T.handle, 0, ptrs, "f32", 8, 6, 0, out.data_ptr())  # ld not a multiple of 8
    assert ei.value.status == P.SPT_EINVAL
    with pytest.raises(P.SptError) as ei:
        P.mttkrp(T.handle, 3, ptrs, "f32", 8, 8, 0, out.data_ptr())
    assert ei.value.status == P.SPT_EINVAL
    with pytest.raises(P.SptError) as ei:
        P.mttkrp(T.handle, 0, ptrs, "f32", 8, 8, 0, out.data_ptr(), P.spt_schedule.make("perm"))
    assert ei.value.status == P.SPT_ESTATE
    with pytest.raises(P.SptError) as ei:
        P.mttkrp(T.handle, 0, ptrs, "f32", 8, 8, 0, out.data_ptr(),
                 P.spt_schedule.make("atomic", lanes_per_nnz=3))
    assert ei.value.status == P.SPT_EINVAL
    T.close()

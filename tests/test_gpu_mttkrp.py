"""GPU parity: MTTKRP through the C ABI vs the FP64 oracle, element by element.

Covers every scatter strategy (atomic, permuted via perm_n, permuted over
the mode-sorted copy, privatised in shared memory), fp32 / bf16 / f16 factors, orders 1-5, ranks that are
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

SCATTERS = ["atomic", "perm", "sorted", "private"]


def _lib():
    import paper_1809_09175_gb300 as P
    return P


def _run(P, idx, vals, dims, facs, dtype, R, scatter, sched_kw=None, lam=None, modes=None):
    T = P.SparseTensor(idx, vals, dims)
    if scatter not in ("atomic", "private"):
        T.build_permutation(-1, index_only=(scatter == "perm"))
    dev = [to_device_factor(f, dtype) for f in facs]
    lam_dt = np.float64 if dtype == "f64" else np.float32
    lam_t = None if lam is None else torch.from_numpy(lam.astype(lam_dt)).cuda()
    outs = {}
    for n in (range(len(dims)) if modes is None else modes):
        sched = None
        if sched_kw is not None or scatter is not None:
            base = P.mttkrp_default_schedule(T.handle, n, dtype, R).as_dict()
            base["scatter"] = P.SCATTERS[scatter]
            base.update(sched_kw or {})
            sched = P.spt_schedule.make(**base)
        try:
            outs[n] = T.mttkrp(n, dev, R, lam=lam_t, sched=sched).cpu().numpy()
        except P.SptError as e:
            # a private copy of this mode's output exceeds 8 CTAs' shared memory
            ab = 8 if dtype == "f64" else 4
            if scatter != "private" or e.status != P.SPT_EINVAL or dims[n] * R * ab < 8 * 100_000:
                raise
            outs[n] = None
    T.check()
    T.close()
    return outs


def _oracle(idx, vals, dims, facs, dtype, R, n, lam=None):
    A = [widen(f, dtype, R) for f in facs]
    if lam is not None:  # the weights as the kernel receives them
        lam = lam.astype(np.float64) if dtype == "f64" else lam.astype(np.float32).astype(np.float64)
    return oracle.mttkrp(idx, vals, dims, A, n, R, lam=lam)


@pytest.mark.parametrize("scatter", SCATTERS)
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "f64"])
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
        assert got is not None
        assert np.all(got[:, R:] == 0)
        e = rel_fro(got[:, :R], ref)
        assert e <= TOL[dtype], (n, e)
        rt = 1e-12 if dtype == "f64" else 1e-5
        np.testing.assert_allclose(got[:, :R], ref, rtol=rt, atol=rt * np.abs(ref).max())


@pytest.mark.parametrize("scatter", SCATTERS)
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "f64"])
def test_integer_case_bit_exact(scatter, dtype):
    P = _lib()
    dims = (300, 200, 50, 7)
    R = 13
    idx, vals, facs = synth.small_integer_case(dims, 40_000, R, 5, dtype=dtype)
    outs = _run(P, idx, vals, dims, facs, dtype, R, scatter, {"nnz_per_group": 9})
    for n in range(4):
        ref = _oracle(idx, vals, dims, facs, dtype, R, n)
        assert np.abs(ref).max() < 2 ** 24
        np.testing.assert_array_equal(outs[n][:, :R], ref.astype(outs[n].dtype))


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
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_schedules_and_ranks(sk, R, dtype):
    P = _lib()
    dims = (5000, 800, 300)
    idx, vals = synth.coo_zipf(dims, 60_003, (1.3, 0.7, 0.0), 9)
    facs = synth.factor_matrices(dims, R, 4, "normal", dtype=dtype)
    for scatter in SCATTERS:
        outs = _run(P, idx, vals, dims, facs, dtype, R, scatter, SCHEDS[sk])
        for n in range(3):
            got = outs[n]
            if got is None:  # private copy too large for this rank (checked in _run)
                continue
            ref = _oracle(idx, vals, dims, facs, dtype, R, n)
            assert np.all(got[:, R:] == 0)
            e = rel_fro(got[:, :R], ref)
            assert e <= (1e-12 if dtype == "f64" else 1e-5), (scatter, n, e)


def test_private_scatter_cluster_sizes():
    """The privatised scatter on modes whose private output copy needs a
    cluster of 1, 2, 4 and 8 CTAs (R = 32: 128 bytes per row), a skewed
    index distribution and a ragged last chunk; bf16 factors too."""
    P = _lib()
    dims = (900, 2500, 5000, 10000)
    R = 32
    idx, vals = synth.coo_zipf(dims, 400_003, (1.4, 1.0, 0.6, 0.0), 31)
    for dtype in ["f32", "bf16"]:
        facs = synth.factor_matrices(dims, R, 8, "normal", dtype=dtype)
        lam = np.linspace(0.5, 1.5, R)
        outs = _run(P, idx, vals, dims, facs, dtype, R, "private", lam=lam)
        for n in range(4):
            assert outs[n] is not None
            ref = _oracle(idx, vals, dims, facs, dtype, R, n, lam=lam)
            assert np.all(outs[n][:, R:] == 0)
            e = rel_fro(outs[n][:, :R], ref)
            assert e <= 1e-5, (dtype, n, e)


def test_private_scatter_rejects_modes_too_long():
    P = _lib()
    dims = (200_000, 50, 40)
    idx, vals = synth.coo_zipf(dims, 10_000, 1.0, 5)
    T = P.SparseTensor(idx, vals, dims)
    facs = [torch.rand((I, 64), device="cuda") for I in dims]
    cands, valid = P.mttkrp_candidates(T.handle, 0, 64)
    assert not any(v for c, v in zip(cands, valid) if c.scatter == P.SPT_SCATTER_PRIVATE)
    _, valid2 = P.mttkrp_candidates(T.handle, 1, 64)
    assert any(v for c, v in zip(cands, valid2) if c.scatter == P.SPT_SCATTER_PRIVATE)
    sched = P.spt_schedule.make("private", lanes_per_nnz=16, chunks=1, nnz_per_group=12, warps_per_cta=8)
    with pytest.raises(P.SptError) as ei:
        T.mttkrp(0, facs, 64, sched=sched)
    assert ei.value.status == P.SPT_EINVAL
    got = T.mttkrp(1, facs, 64, sched=sched).cpu().numpy()
    A = [f.cpu().numpy().astype(np.float64) for f in facs]
    ref = oracle.mttkrp(idx, vals, dims, A, 1, 64)
    assert rel_fro(got, ref) <= 1e-5
    T.close()


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


@pytest.mark.parametrize("scatter", SCATTERS)
def test_fp64_factors_zipf_orders_3_to_5(scatter):
    """fp64 factors, accumulation and output (the paper's precision) on
    skewed tensors of orders 3-5 and ranks up to 256 (two rank blocks of
    128 columns), with weights."""
    P = _lib()
    for order, R in [(3, 8), (4, 96), (5, 33), (3, 256)]:
        dims = [2000, 900, 500, 64, 9][:order]
        idx, vals = synth.coo_zipf(dims, 50_001, 1.1, 40 + order)
        facs = synth.factor_matrices(dims, R, 6, "normal", dtype="f64")
        lam = np.linspace(0.5, 2.0, R)
        outs = _run(P, idx, vals, dims, facs, "f64", R, scatter, lam=lam)
        for n in range(order):
            if outs[n] is None:
                continue
            assert outs[n].dtype == np.float64
            ref = _oracle(idx, vals, dims, facs, "f64", R, n, lam=lam)
            assert np.all(outs[n][:, R:] == 0)
            e = rel_fro(outs[n][:, :R], ref)
            assert e <= 1e-12, (order, R, n, e)


def test_fp64_outside_mttkrp_is_unsupported():
    P = _lib()
    dims = (30, 20, 10)
    idx, vals = synth.coo_zipf(dims, 1000, 0.5, 2)
    T = P.SparseTensor(idx, vals, dims, coalesce=True)
    facs = [torch.rand((I, 8), dtype=torch.float64, device="cuda") for I in dims]
    lam = torch.zeros(8, dtype=torch.float64, device="cuda")
    ws = T.cp_als_workspace(8, 8)
    with pytest.raises(P.SptError) as ei:
        T.cp_als_step(facs, 8, lam, None, ws)
    assert ei.value.status == P.SPT_EUNSUPPORTED
    T.close()


def _hot_row_tensor(dims, nnz, hot, seed):
    """Uniform coordinates, except that `hot` nonzeros at random storage
    positions share mode-0 row 7 (a row far hotter than any real-world slice
    of this size: every atomic flush of it lands on one output row)."""
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, I, nnz) for I in dims]).astype(np.int32)
    idx[0, rng.choice(nnz, hot, replace=False)] = 7
    return idx, rng.uniform(0.0, 1.0, nnz).astype(np.float32)


@pytest.mark.parametrize("scatter", SCATTERS)
@pytest.mark.parametrize("dist,R", [("normal", 16), ("uniform", 32)])
def test_row_with_two_million_nonzeros(scatter, dist, R):
    """One row holds 2.2e6 of 3e6 nonzeros in random storage order: every
    scatter (the atomic one adds such a row through its shared-memory copy
    of the hot rows) must stay within the fp32 gate on every mode."""
    P = _lib()
    dims = (5000, 3000, 2000)
    idx, vals = _hot_row_tensor(dims, 3_000_000, 2_200_000, 31)
    facs = synth.factor_matrices(dims, R, 31, dist)
    outs = _run(P, idx, vals, dims, facs, "f32", R, scatter)
    for n in range(3):
        if outs[n] is None:
            continue
        ref = _oracle(idx, vals, dims, facs, "f32", R, n)
        err = rel_fro(outs[n][:, :R], ref)
        assert err <= TOL["f32"], (n, err)
        if n == 0:  # the hot row by itself
            assert rel_fro(outs[n][7, :R], ref[7]) <= TOL["f32"], n


@pytest.mark.parametrize("scatter", ["private", "atomic"])
def test_clustered_private_copy_with_a_row_of_six_million_nonzeros(scatter):
    """A 20000-row mode at R = 16 (a 1.28 MB private copy: clusters of 8
    CTAs, about 19 resident at once) whose row 7 holds 6e6 of 2e7 nonzeros in
    random storage order.  One resident wave would add ~3e5 values into that
    row of each cluster's copy; the private scatter runs more, shorter waves
    of clusters instead and must stay within the fp32 gate, and so must the
    atomic scatter (hot-row copy in shared memory)."""
    P = _lib()
    dims = (20_000, 3000, 2000)
    R = 16
    idx, vals = _hot_row_tensor(dims, 20_000_000, 6_000_000, 41)
    facs = synth.factor_matrices(dims, R, 41, "uniform")
    outs = _run(P, idx, vals, dims, facs, "f32", R, scatter, modes=[0])
    ref = _oracle(idx, vals, dims, facs, "f32", R, 0)
    assert rel_fro(outs[0][:, :R], ref) <= TOL["f32"]
    assert rel_fro(outs[0][7, :R], ref[7]) <= TOL["f32"]


@pytest.mark.parametrize("order", [3, 4, 5])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_slice_ordered_copy_and_single_row_chunks(order, dtype):
    """Mode-sorted copies built with SPT_PERM_SLICE_ORDER (each slice ordered
    by the next modes) and power-law rows long enough that whole chunks lie in
    one row (those take the consecutive-nonzero walk): every mode against the
    oracle, for several chunk shapes, and the deterministic call bit-identical
    from call to call."""
    P = _lib()
    dims = {3: (400, 300, 200), 4: (300, 200, 100, 50), 5: (200, 150, 100, 50, 20)}[order]
    R = 24
    idx, vals = synth.coo_zipf(dims, 200_000, 1.3, 40 + order)
    facs = synth.factor_matrices(dims, R, 40 + order, "normal", dtype=dtype)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation(slice_order=True)
    dev = [to_device_factor(f, dtype) for f in facs]
    for n in range(order):
        ref = _oracle(idx, vals, dims, facs, dtype, R, n)
        for S_, lanes, warps in [(7, 8, 4), (23, 8, 8), (63, 4, 8)]:
            sc = P.spt_schedule.make("sorted", lanes_per_nnz=lanes, chunks=1 if lanes * 4 >= R else 2,
                                     nnz_per_group=S_, warps_per_cta=warps)
            got = T.mttkrp(n, dev, R, sched=sc).cpu().numpy()[:, :R]
            assert rel_fro(got, ref) <= TOL[dtype], (n, S_, lanes)
        a = T.mttkrp(n, dev, R, deterministic=True).cpu().numpy()
        b = T.mttkrp(n, dev, R, deterministic=True).cpu().numpy()
        np.testing.assert_array_equal(a, b)
        assert rel_fro(a[:, :R], ref) <= TOL[dtype]
    T.check()
    T.close()


@pytest.mark.parametrize("R", [32, 48, 64])
def test_atomic_scatter_on_a_short_mode_with_long_rows(R):
    """A 100-row mode holding 3e7 nonzeros (3e5 per row, storage order
    random).  The hot-row copy in shared memory holds 64 (R=64), 85 (R=48)
    or all 100 (R=32) rows; every other row takes its 3e5 adds in global
    memory, where one fp32 chain of that length drifts by a few 1e-5
    relative (U(0,1) factors: the sums only grow).  The scatter splits those
    adds over copies of the output and must stay within the fp32 gate."""
    P = _lib()
    import os
    dims = (100, 5000, 4000)
    rng = np.random.default_rng(77)
    nnz = 30_000_000
    idx = np.stack([rng.integers(0, I, nnz) for I in dims]).astype(np.int32)
    vals = rng.uniform(0.0, 1.0, nnz).astype(np.float32)
    facs = synth.factor_matrices(dims, R, 77, "uniform")
    T = P.SparseTensor(idx, vals, dims)
    dev = [to_device_factor(f, "f32") for f in facs]
    base = P.mttkrp_default_schedule(T.handle, 0, "f32", R).as_dict()
    base["scatter"] = P.SPT_SCATTER_ATOMIC
    got = T.mttkrp(0, dev, R, sched=P.spt_schedule.make(**base)).cpu().numpy()[:, :R]
    T.check()
    T.close()
    ref = oracle.mttkrp_threads(idx, vals, dims, [widen(f, "f32", R) for f in facs], 0, R, os.cpu_count() or 4)
    assert rel_fro(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("order", [3, 4])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_l2_blocked_copy(order, dtype):
    """The sorted traversal over an L2-blocked copy (one launch per block of
    the longest other mode's rows, each adding the rows it owns): every mode
    against the oracle for blocks of 1 row (many empty groups), 97 rows
    (ragged groups with padding records) and 1000 rows, two chunk shapes;
    dropping the copy restores the plain traversal; the deterministic call
    keeps the plain copy; bad arguments are refused."""
    P = _lib()
    dims = {3: (3000, 200, 150), 4: (2500, 120, 60, 30)}[order]
    R = 20
    idx, vals = synth.coo_zipf(dims, 150_000, 1.0, 80 + order)
    facs = synth.factor_matrices(dims, R, 80 + order, "normal", dtype=dtype)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation(slice_order=True)
    dev = [to_device_factor(f, dtype) for f in facs]
    for n in range(order):
        ref = _oracle(idx, vals, dims, facs, dtype, R, n)
        bm = max((m for m in range(order) if m != n), key=lambda m: dims[m])
        for rows in (1, 97, 1000):
            T.build_l2_blocks(n, -1, rows)
            assert T.l2_blocks(n) == (bm, rows, -(-dims[bm] // rows))
            for S_, lanes, warps in [(7, 8, 4), (23, 4, 8)]:
                sc = P.spt_schedule.make("sorted", lanes_per_nnz=lanes, chunks=1 if lanes * 4 >= R else 2,
                                         nnz_per_group=S_, warps_per_cta=warps)
                got = T.mttkrp(n, dev, R, sched=sc).cpu().numpy()
                assert rel_fro(got[:, :R], ref) <= TOL[dtype], (n, rows, S_, lanes)
                assert np.all(got[:, R:] == 0)
        det = T.mttkrp(n, dev, R, deterministic=True).cpu().numpy()[:, :R]
        assert rel_fro(det, ref) <= TOL[dtype]
        T.build_l2_blocks(n, block_rows=0)
        assert T.l2_blocks(n)[0] == -1
        assert rel_fro(T.mttkrp(n, dev, R).cpu().numpy()[:, :R], ref) <= TOL[dtype]
    with pytest.raises(P.SptError):
        T.build_l2_blocks(0, 0, 10)  # the blocked mode is the mode itself
    T.check()
    T.close()
    T2 = P.SparseTensor(idx, vals, dims)
    T2.build_permutation(index_only=True)
    with pytest.raises(P.SptError) as e:
        T2.build_l2_blocks(0)  # no mode-sorted copy
    assert e.value.status == P.SPT_ESTATE
    T2.close()


@pytest.mark.parametrize("order", [2, 3, 4, 5])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_perm_traversal_over_storage_records(order, dtype):
    """The perm_n traversal (Fig. MTTKRP-C) reading one storage-order record
    per nonzero (`tensor_storage_records`: 4-word records for orders 2-3,
    6-word ones for 4-5) against the oracle on every mode, two chunk shapes,
    and against the same traversal over the separate coordinate arrays (the
    same tensor once the records are dropped)."""
    P = _lib()
    dims = {2: (700, 500), 3: (400, 300, 200), 4: (300, 200, 100, 50), 5: (200, 150, 100, 50, 20)}[order]
    R = 20
    idx, vals = synth.coo_zipf(dims, 60_000, 1.1, 90 + order)
    facs = synth.factor_matrices(dims, R, 90 + order, "normal", dtype=dtype)
    dev = [to_device_factor(f, dtype) for f in facs]
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation(index_only=True)
    scheds = [P.spt_schedule.make("perm", lanes_per_nnz=lanes, chunks=1 if lanes * 4 >= R else 2,
                                  nnz_per_group=S_, warps_per_cta=4) for S_, lanes in [(7, 8), (23, 4)]]
    T.storage_records()
    T.storage_records()  # a second call keeps the records
    got = [[T.mttkrp(n, dev, R, sched=sc).cpu().numpy() for sc in scheds] for n in range(order)]
    T.storage_records(False)
    plain = [[T.mttkrp(n, dev, R, sched=sc).cpu().numpy() for sc in scheds] for n in range(order)]
    for n in range(order):
        ref = _oracle(idx, vals, dims, facs, dtype, R, n)
        for k in range(len(scheds)):
            assert rel_fro(got[n][k][:, :R], ref) <= TOL[dtype], (n, k)
            assert rel_fro(got[n][k][:, :R], plain[n][k][:, :R]) <= TOL[dtype]
    with pytest.raises(P.SptError):
        P.tensor_storage_records(T.handle, 2)
    T.check()
    T.close()

"""GPU parity: CP-ALS iterations through the C ABI vs the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import rel_fro, to_device_factor

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1809_09175_gb300 as P
    return P


def _setup(P, idx, vals, dims, R, facs_np, dtype="f32"):
    T = P.SparseTensor(idx, vals, dims, coalesce=True)
    T.build_permutation()
    facs = [to_device_factor(f, dtype) for f in facs_np]
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = T.cp_als_workspace(R, facs[0].shape[1])
    return T, facs, lam, fit, ws


def _fac64(t, R):
    return t.float().cpu().numpy()[:, :R].astype(np.float64)


# One CP-ALS step (every mode once) from the same starting factors.  The
# gate is the FP32 bound of 1e-5 relative Frobenius error wherever the
# arithmetic allows it.  The GPU's fp32 steps -- V from the fp32 MTTKRP (its
# own rounding plus the accumulation, ~2 units of u = 2^-24 measured), the
# Grams' fp32 partial sums folded into FP64 (~2u), H^-1 rounded to fp32 and
# the fp32 apply V H^-1 -- perturb V and H by a few u relative, and the
# solve of A H = V turns relative perturbations eps of V and H into at most
# cond(H) * eps in A (first order).  So mode n is held to
#     max(1e-5, 4 cond(H_n) u)
# with H_n the oracle's Gram-Hadamard matrix of that mode.  A float32
# simulation of the same steps on the 100x80x60 case (cond(H) = 44, 5.1, 3.1)
# gives 1.4e-6, 8e-7, 8e-7; on the 3-way power-law case below mode 2 has
# cond(H) = 5.4e4, where rounding V once to fp32 already gives 4.4e-4.
U32 = 2.0 ** -24


def _gram_hadamard_conds(A_old, A_new):
    """cond(H_n) for n = 0..d-1 along the oracle's step: modes before n are
    already updated, modes after n still hold the starting factors."""
    d = len(A_old)
    conds = []
    for n in range(d):
        H = np.ones((A_old[0].shape[1],) * 2)
        for m in range(d):
            if m != n:
                f = A_new[m] if m < n else A_old[m]
                H *= f.T @ f
        conds.append(float(np.linalg.cond(H)))
    return conds


def _one_step(P, idx, vals, dims, R, facs_np, block_rows=None):
    T, facs, lam, fit, ws = _setup(P, idx, vals, dims, R, facs_np)
    if block_rows is not None:  # every mode's sorted traversal over its L2-blocked copy
        for m in range(len(dims)):
            T.build_l2_blocks(m, -1, block_rows)
    A = [f[:, :R].astype(np.float64).copy() for f in facs_np]
    A_old = [a.copy() for a in A]
    T.cp_als_step(facs, R, lam, fit, ws)
    P.cp_als_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    c_idx, c_vals = T.coo()  # the coalesced nonzeros the GPU works on
    c_idx, c_vals = c_idx.cpu().numpy(), c_vals.cpu().numpy()
    lam_o, fit_o, st = oracle.cp_als_iter(c_idx, c_vals, dims, A, R)
    assert st == 0
    errs = [rel_fro(_fac64(facs[m], R), A[m]) for m in range(len(dims))]
    tols = [max(1e-5, 4.0 * c * U32) for c in _gram_hadamard_conds(A_old, A)]
    for m in range(len(dims)):
        assert errs[m] <= tols[m], (m, errs, tols)
    # lambda holds the last mode's column norms, the fit its residual
    assert rel_fro(lam.cpu().numpy(), lam_o) <= tols[-1]
    assert abs(float(fit.item()) - fit_o) <= tols[-1]
    T.close()
    return errs, tols


def test_one_step_matches_oracle_uniform_100x80x60():
    P = _lib()
    w = synth.WORKLOADS["uniform3d_100x80x60_nnz1e4"]
    idx, vals = w.coo()
    errs, tols = _one_step(P, idx, vals, w.dims, w.R, w.factors())
    assert max(tols) <= 1.1e-5  # well conditioned: the plain 1e-5 gate applies


@pytest.mark.parametrize("dims,nnz,s,R,seed", [((3000, 2000, 1000), 400_000, 1.1, 32, 5),
                                               ((500, 400, 300, 200), 300_000, 0.8, 16, 6)])
def test_one_step_matches_oracle_power_law(dims, nnz, s, R, seed):
    P = _lib()
    idx, vals = synth.coo_zipf(dims, nnz, s, seed)
    _one_step(P, idx, vals, dims, R, synth.factor_matrices(dims, R, seed, "uniform"))


def test_one_step_over_l2_blocked_copies():
    """CP-ALS whose MTTKRPs run over L2-blocked copies (blocks of 37 rows of
    the longest other mode: one launch per block, rows added across
    launches) meets the same one-step gates against the oracle."""
    P = _lib()
    dims = (600, 500, 400)
    idx, vals = synth.coo_zipf(dims, 120_000, 1.0, 21)
    facs_np = synth.factor_matrices(dims, 16, 21, "uniform")
    _one_step(P, idx, vals, dims, 16, facs_np, block_rows=37)


def test_ten_iterations_fit_trajectory():
    P = _lib()
    w = synth.WORKLOADS["uniform3d_100x80x60_nnz1e4"]
    idx, vals = w.coo()
    R = w.R
    facs_np = w.factors()
    T, facs, lam, fit, ws = _setup(P, idx, vals, w.dims, R, facs_np)
    A = [f[:, :R].astype(np.float64).copy() for f in facs_np]
    x2 = oracle.norm2(idx, vals)
    assert abs(T.norm2() - x2) <= 1e-9 * x2
    for it in range(10):
        T.cp_als_step(facs, R, lam, fit, ws)
        _, fit_o, st = oracle.cp_als_iter(idx, vals, w.dims, A, R, xnorm2=x2)
        assert st == 0
        assert abs(float(fit.item()) - fit_o) <= 1e-4, (it, float(fit.item()), fit_o)
    T.close()


def test_recovers_exact_rank3_tensor():
    P = _lib()
    from tests.test_oracle_pins import _sparse_ktensor
    dims = (30, 20, 10)
    R = 3
    idx, vals, truth = _sparse_ktensor(dims, R, 0)
    rng = np.random.default_rng(100)
    ld = 8
    facs_np = []
    for I in dims:
        f = np.zeros((I, ld), np.float32)
        f[:, :R] = rng.uniform(0, 1, (I, R))
        facs_np.append(f)
    T, facs, lam, fit, ws = _setup(P, idx, vals.astype(np.float32), dims, R, facs_np)
    for _ in range(200):
        T.cp_als_step(facs, R, lam, fit, ws)
    assert float(fit.item()) > 0.999
    # each true component is matched by a computed one (congruence ~ 1)
    for m in range(3):
        Fm = _fac64(facs[m], R)
        Tm = truth[m] / np.linalg.norm(truth[m], axis=0)
        C = np.abs(Tm.T @ Fm)
        assert (C.max(axis=1) > 0.999).all(), C
    T.close()


def test_bf16_one_step_within_2e3():
    P = _lib()
    dims = (400, 300, 200)
    idx, vals = synth.coo_zipf(dims, 60_000, 0.8, 3)
    R = 16
    facs_np = synth.factor_matrices(dims, R, 3, "uniform", dtype="bf16")
    T, facs, lam, fit, ws = _setup(P, idx, vals, dims, R, facs_np, "bf16")
    A = [oracle.as_f64(f, "bf16")[:, :R].copy() for f in facs_np]
    T.cp_als_step(facs, R, lam, fit, ws)
    lam_o, fit_o, st = oracle.cp_als_iter(idx, vals, dims, A, R, bf16=True)
    errs = [rel_fro(_fac64(facs[m], R), A[m]) for m in range(3)]
    assert max(errs) <= 2e-3, errs
    assert abs(float(fit.item()) - fit_o) <= 2e-3
    T.close()


def test_singular_and_state_errors():
    P = _lib()
    dims = (20, 10, 8)
    idx, vals = synth.coo_uniform_distinct(dims, 300, 1)
    R = 4
    facs_np = [np.zeros((I, 8), np.float32) for I in dims]
    T, facs, lam, fit, ws = _setup(P, idx, vals, dims, R, facs_np)
    T.cp_als_step(facs, R, lam, fit, ws)
    with pytest.raises(P.SptError) as ei:
        P.cp_als_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == P.SPT_ESINGULAR
    T.close()
    T2 = P.SparseTensor(idx, vals, dims)  # not coalesced
    with pytest.raises(P.SptError) as ei:
        P.cp_als_step(T2.handle, [f.data_ptr() for f in facs], "f32", R, 8, lam.data_ptr(), 0,
                      ws.data_ptr(), ws.numel())
    assert ei.value.status == P.SPT_ESTATE
    with pytest.raises(P.SptError) as ei:
        P.cp_als_workspace_size(T2.handle, 129, 136)
    assert ei.value.status == P.SPT_EUNSUPPORTED
    T2.close()


def test_graph_replay_matches_direct_launch_and_resume():
    """Captured-graph replay on a side stream vs direct launches on the legacy
    stream: one iteration gives the same factors (to the rounding of the
    unordered atomic adds); a run checkpointed to host and resumed in new
    buffers follows the same fit trajectory.  (Later iterates are compared
    through the fit: ALS amplifies the rounding-level differences of the
    atomic order in the factors themselves.)"""
    P = _lib()
    dims = (500, 400, 300, 20)
    idx, vals = synth.coo_zipf(dims, 80_000, 1.1, 5)
    R = 24
    # N(0,1) starting factors keep the Gram-Hadamard systems well conditioned,
    # so the comparison measures replay equivalence, not conditioning
    facs_np = synth.factor_matrices(dims, R, 5, "normal")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        T, facs, lam, fit, ws = _setup(P, idx, vals, dims, R, facs_np)
        fits_graph = []
        for it in range(5):
            T.cp_als_step(facs, R, lam, fit, ws)
            fits_graph.append(float(fit.item()))
            if it == 0:
                first = [f.clone() for f in facs]
    torch.cuda.synchronize()
    T2, facs2, lam2, fit2, ws2 = _setup(P, idx, vals, dims, R, facs_np)

    def direct(fs):
        P.cp_als_step(T2.handle, [f.data_ptr() for f in fs], "f32", R, fs[0].shape[1],
                      lam2.data_ptr(), fit2.data_ptr(), ws2.data_ptr(), ws2.numel(), 0)
        torch.cuda.synchronize()
        return float(fit2.item())

    fits = [direct(facs2)]
    for a, b in zip(first, facs2):
        # two runs differ only in the order of float atomic adds (~1e-7),
        # amplified by the four Gram-Hadamard solves of the iteration
        assert rel_fro(b.cpu().numpy(), a.cpu().numpy()) <= 1e-4
    fits += [direct(facs2) for _ in range(2)]
    ckpt = [f.cpu() for f in facs2]
    facs3 = [c.cuda() for c in ckpt]
    fits += [direct(facs3) for _ in range(2)]
    np.testing.assert_allclose(fits, fits_graph, rtol=0, atol=1e-6)
    T.close()
    T2.close()

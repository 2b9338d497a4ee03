"""GPU parity: the generalised CP gradient (gcp_gradient) against the FP64
oracle's definition, for the Poisson (every entry of the tensor),
Bernoulli-logit and Gaussian (stored entries) losses, orders 3-5, ranks
within one and two lane chunks per lane, fp32 and bf16 factors."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import rel_fro, to_device_factor, widen

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1809_09175_gb300 as P
    return P


def _case(order, R, loss, dtype, seed):
    dims = [900, 700, 300, 40, 7][:order]
    idx, vals = synth.coo_zipf(dims, 60_001, 1.1, seed)
    if loss == "bernoulli":
        vals = (vals > 0.6).astype(np.float32)  # binary data, stored zeros included
    facs = synth.factor_matrices(dims, R, seed, "uniform", dtype=dtype)
    if loss == "poisson":  # keep m > 0 away from zero
        facs = synth.factor_matrices(dims, R, seed, "uniform", dtype="f32")
        facs = [np.where(np.arange(f.shape[1]) < R, f + 0.05, 0.0).astype(np.float32) for f in facs]
        if dtype == "bf16":
            facs = [synth._to_bf16_bits(f) for f in facs]
    return dims, idx, vals, facs


@pytest.mark.parametrize("loss", ["poisson", "bernoulli", "gaussian"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("order,R", [(3, 16), (4, 20), (5, 8), (3, 100)])
def test_gcp_gradient_matches_oracle(loss, dtype, order, R):
    P = _lib()
    dims, idx, vals, facs = _case(order, R, loss, dtype, 50 + order)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    dev = [to_device_factor(f, dtype) for f in facs]
    A = [widen(f, dtype, R) for f in facs]
    for n in range(order):
        G, F = T.gcp_gradient(n, dev, R, loss)
        Gr, Fr = oracle.gcp_grad(idx, vals, dims, A, n, R, loss)
        got = G.cpu().numpy()
        assert np.all(got[:, R:] == 0)
        e = rel_fro(got[:, :R], Gr)
        assert e <= 2e-5, (loss, dtype, order, R, n, e)
        assert abs(float(F.item()) - Fr) <= 1e-5 * abs(Fr), (float(F.item()), Fr)
    T.check()
    T.close()


def test_gcp_gaussian_on_full_tensor_is_normal_equation_residual():
    """Every coordinate stored once: the Gaussian gradient equals
    2 (A^(n) H - MTTKRP), H the Hadamard product of the other Grams."""
    P = _lib()
    dims = (30, 20, 10)
    R = 8
    grid = np.stack(np.meshgrid(*[np.arange(I) for I in dims], indexing="ij")).reshape(3, -1)
    rng = np.random.default_rng(4)
    perm = rng.permutation(grid.shape[1])
    idx = np.ascontiguousarray(grid[:, perm].astype(np.int32))
    vals = rng.random(idx.shape[1]).astype(np.float32)
    facs = synth.factor_matrices(dims, R, 2, "normal")
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    dev = [to_device_factor(f, "f32") for f in facs]
    for n in range(3):
        G, _ = T.gcp_gradient(n, dev, R, "gaussian")
        H = np.ones((R, R))
        for l in range(3):
            if l != n:
                H *= facs[l][:, :R].astype(np.float64).T @ facs[l][:, :R].astype(np.float64)
        V = T.mttkrp(n, dev, R).cpu().numpy()[:, :R].astype(np.float64)
        ref = 2 * (facs[n][:, :R].astype(np.float64) @ H - V)
        assert rel_fro(G.cpu().numpy()[:, :R], ref) <= 1e-4
    T.close()


def test_gcp_errors():
    P = _lib()
    dims = (30, 20, 10)
    idx, vals = synth.coo_zipf(dims, 500, 0.5, 1)
    T = P.SparseTensor(idx, vals, dims)
    dev = [torch.rand((I, 8), device="cuda") for I in dims]
    with pytest.raises(P.SptError) as ei:  # no mode-sorted copy yet
        T.gcp_gradient(0, dev, 8, "poisson")
    assert ei.value.status == P.SPT_ESTATE
    T.build_permutation()
    with pytest.raises(P.SptError) as ei:
        T.gcp_gradient(0, [f.double() for f in dev], 8, "poisson")
    assert ei.value.status == P.SPT_EUNSUPPORTED
    T.close()

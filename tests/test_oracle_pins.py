"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks an oracle routine against the mathematics: the dense
matricized definition, a library sparse product, closed forms, exact integer
arithmetic, invariants, brute force on tiny inputs, or recovery of a known
CP model.  None of them re-types the oracle's own loop.
"""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle
import synth


def _dense(idx, vals, dims):
    X = np.zeros(dims)
    np.add.at(X, tuple(idx.astype(np.int64)), vals.astype(np.float64))
    return X


def _khatri_rao_unfold_mttkrp(X, factors, n, R):
    """V = X_(n) (A^(d) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1)), the
    matricized form of MTTKRP (Kolda-Bader ordering: lower modes vary fastest)."""
    d = X.ndim
    In = X.shape[n]
    Xn = np.moveaxis(X, n, 0).reshape(In, -1, order="F")
    others = [m for m in range(d) if m != n]
    KR = np.empty((Xn.shape[1], R))
    for j in range(R):
        col = np.ones(1)
        for m in others:  # kron(a_m, col): the new (higher) mode varies slowest
            col = np.kron(factors[m][:, j], col)
        KR[:, j] = col
    return Xn @ KR


@pytest.mark.parametrize("dims,nnz,R,seed", [
    ((7, 5, 6), 60, 4, 1),
    ((4, 6, 3, 5), 80, 3, 2),
    ((3, 4, 2, 3, 2), 40, 5, 3),
])
def test_mttkrp_matches_dense_unfolding(dims, nnz, R, seed):
    idx, vals = synth.coo_uniform(dims, nnz, seed)  # duplicates allowed (additive)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, seed, "normal")]
    lam = np.random.default_rng(seed).uniform(0.5, 2.0, R)
    X = _dense(idx, vals, dims)
    for n in range(len(dims)):
        ref = _khatri_rao_unfold_mttkrp(X, facs, n, R) * lam[None, :]
        got = oracle.mttkrp(idx, vals, dims, facs, n, R, lam=lam)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_mttkrp_order2_is_spmm():
    import scipy.sparse as sp
    dims = (40, 30)
    idx, vals = synth.coo_uniform(dims, 300, 5)
    R = 6
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 5, "normal")]
    X = sp.coo_matrix((vals.astype(np.float64), (idx[0], idx[1])), shape=dims).tocsr()
    np.testing.assert_allclose(oracle.mttkrp(idx, vals, dims, facs, 0, R), X @ facs[1],
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.mttkrp(idx, vals, dims, facs, 1, R), X.T @ facs[0],
                               rtol=1e-12, atol=1e-12)


def test_single_nonzero_closed_form():
    dims = (5, 4, 3)
    idx = np.array([[3], [1], [2]], dtype=np.int32)
    vals = np.array([2.5], dtype=np.float32)
    R = 3
    facs = [np.arange(I * R, dtype=np.float64).reshape(I, R) + 1 for I in dims]
    for n in range(3):
        V = oracle.mttkrp(idx, vals, dims, facs, n, R)
        expect = np.zeros((dims[n], R))
        row = 2.5 * np.ones(R)
        for m in range(3):
            if m != n:
                row = row * facs[m][idx[m, 0]]
        expect[idx[n, 0]] = row
        np.testing.assert_array_equal(V, expect)


def test_all_ones_factors_give_slice_sums():
    dims = (20, 15, 10)
    idx, vals = synth.coo_uniform(dims, 500, 9)
    R = 4
    facs = [np.ones((I, R)) for I in dims]
    for n in range(3):
        V = oracle.mttkrp(idx, vals, dims, facs, n, R)
        sums = np.bincount(idx[n], weights=vals.astype(np.float64), minlength=dims[n])
        np.testing.assert_allclose(V, np.repeat(sums[:, None], R, axis=1), rtol=1e-13)


def test_integer_case_is_exact():
    dims = (30, 20, 10, 7)
    idx, vals, facs = synth.small_integer_case(dims, 2000, 5, 11)
    R = 5
    F = [f[:, :R].astype(np.int64) for f in facs]
    for n in range(4):
        prod = vals.astype(np.int64)[:, None] * np.ones((1, R), dtype=np.int64)
        for m in range(4):
            if m != n:
                prod = prod * F[m][idx[m]]
        exact = np.zeros((dims[n], R), dtype=np.int64)
        np.add.at(exact, idx[n], prod)
        got = oracle.mttkrp(idx, vals, dims, [f.astype(np.float64) for f in F], n, R)
        np.testing.assert_array_equal(got, exact.astype(np.float64))


def test_linearity_and_order_invariance():
    dims = (12, 9, 8)
    R = 4
    i1, v1 = synth.coo_uniform(dims, 200, 21)
    i2, v2 = synth.coo_uniform(dims, 150, 22)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 21, "normal")]
    a, b = 0.75, -2.0  # exact in binary, so the scaled values are exact
    idx = np.concatenate([i1, i2], axis=1)
    vals = np.concatenate([a * v1.astype(np.float64), b * v2.astype(np.float64)])
    perm = np.random.default_rng(0).permutation(idx.shape[1])
    for n in range(3):
        lhs = oracle.mttkrp(idx, vals, dims, facs, n, R)
        rhs = a * oracle.mttkrp(i1, v1, dims, facs, n, R) + b * oracle.mttkrp(i2, v2, dims, facs, n, R)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
        shuf = oracle.mttkrp(idx[:, perm], vals[perm], dims, facs, n, R)
        np.testing.assert_allclose(shuf, lhs, rtol=1e-12, atol=1e-12)


def test_mttkrp_rows_matches_full():
    dims = (50, 40, 30)
    R = 6
    idx, vals = synth.coo_zipf(dims, 3000, 1.1, 4)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 4, "normal")]
    lam = np.linspace(0.5, 1.5, R)
    rows = np.array([0, 7, 7, 49, 13], dtype=np.int32)
    for n in range(3):
        full = oracle.mttkrp(idx, vals, dims, facs, n, R, lam=lam)
        r = rows[rows < dims[n]]
        np.testing.assert_array_equal(oracle.mttkrp_rows(idx, vals, dims, facs, n, R, r, lam=lam),
                                      full[r])


@pytest.mark.parametrize("T", [1, 3, 8, 64])
def test_mttkrp_threads_matches_dense_unfolding(T):
    """The all-core form against the dense X_(n) (Khatri-Rao) product, and
    bit for bit against the serial definition (each row gets the same adds in
    the same order); T = 64 exceeds the rows and nonzeros of the second case,
    a hot row takes most nonzeros of the third."""
    dims = (9, 7, 5)
    R = 4
    idx, vals = synth.coo_uniform(dims, 150, 33)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 33, "normal")]
    X = _dense(idx, vals, dims)
    lam = np.linspace(0.5, 1.5, R)
    for n in range(3):
        got = oracle.mttkrp_threads(idx, vals, dims, facs, n, R, T, lam=lam)
        ref = _khatri_rao_unfold_mttkrp(X, facs, n, R) * lam
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(got, oracle.mttkrp(idx, vals, dims, facs, n, R, lam=lam))
    dims = (6, 5, 4, 3)
    idx, vals, F = synth.small_integer_case(dims, 40, 3, 12)
    F = [f[:, :3].astype(np.float64) for f in F]
    for n in range(4):
        np.testing.assert_array_equal(oracle.mttkrp_threads(idx, vals, dims, F, n, 3, T),
                                      oracle.mttkrp(idx, vals, dims, F, n, 3))
    dims = (40, 30, 20)
    idx, vals = synth.coo_zipf(dims, 5000, (2.5, 1.0, 0.0), 13)
    facs = [f[:, :R].astype(np.float64) for f in synth.factor_matrices(dims, R, 13, "normal")]
    for n in range(3):
        np.testing.assert_array_equal(oracle.mttkrp_threads(idx, vals, dims, facs, n, R, T),
                                      oracle.mttkrp(idx, vals, dims, facs, n, R))
    empty = oracle.mttkrp_threads(np.zeros((3, 0), np.int32), np.zeros(0), (4, 3, 2),
                                  [np.ones((I, 2)) for I in (4, 3, 2)], 0, 2, T)
    assert empty.shape == (4, 2) and not empty.any()


def test_stable_argsort_brute_force():
    rng = np.random.default_rng(3)
    for P, K in [(0, 3), (1, 1), (50, 3), (500, 40), (2000, 2000)]:
        keys = rng.integers(0, K, size=P).astype(np.int32)
        ref = sorted(range(P), key=lambda i: (int(keys[i]), i))
        np.testing.assert_array_equal(oracle.stable_argsort(keys), np.array(ref, dtype=np.int32))
        np.testing.assert_array_equal(oracle.stable_argsort(keys), np.argsort(keys, kind="stable"))


def test_coalesce_brute_force():
    dims = (6, 5, 4)
    idx, vals = synth.coo_zipf(dims, 400, 1.5, 8)
    acc = {}
    for i in range(idx.shape[1]):
        key = tuple(int(x) for x in idx[:, i])
        acc[key] = acc.get(key, 0.0) + float(vals[i])
    keys = sorted(acc)
    ci, cv = oracle.coalesce(idx, vals)
    assert ci.shape[1] == len(keys)
    np.testing.assert_array_equal(ci.T, np.array(keys, dtype=np.int32))
    np.testing.assert_allclose(cv, [acc[k] for k in keys], rtol=1e-15)
    X = _dense(idx, vals, dims)
    assert abs(oracle.norm2(idx, vals) - float((X * X).sum())) < 1e-12 * float((X * X).sum())


def test_gram_and_cholesky():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 12))
    G = oracle.gram(A)
    np.testing.assert_allclose(G, A.T @ A, rtol=1e-12, atol=1e-12)
    L = oracle.cholesky(G)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.linalg.norm(L @ L.T - G) <= 1e-13 * np.linalg.norm(G)
    np.testing.assert_allclose(L, np.linalg.cholesky(G), rtol=1e-10, atol=1e-12)
    # not positive definite -> None
    B = rng.standard_normal((5, 8))
    assert oracle.cholesky(B.T @ B) is None
    assert oracle.cholesky(-np.eye(3)) is None


def _sparse_ktensor(dims, R, seed, density=0.35):
    """Rank-R model whose factors have sparse support, densified to COO."""
    rng = np.random.default_rng(seed)
    facs = []
    for I in dims:
        A = rng.uniform(0.5, 1.5, (I, R)) * (rng.random((I, R)) < density)
        for j in range(R):  # every column has support
            if not A[:, j].any():
                A[rng.integers(I), j] = 1.0
        facs.append(A)
    X = np.einsum("ir,jr,kr->ijk", *facs)
    nz = np.nonzero(X)
    idx = np.stack(nz).astype(np.int32)
    vals = X[nz]
    return idx, vals, facs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cp_als_recovers_exact_rank_r_tensor(seed):
    dims = (30, 20, 10)
    R = 3
    idx, vals, _ = _sparse_ktensor(dims, R, seed)
    # values stored exactly as float64 here (the oracle takes float64)
    rng = np.random.default_rng(100 + seed)
    A = [rng.uniform(0, 1, (I, R)) for I in dims]
    x2 = float((vals * vals).sum())
    fits = []
    for it in range(200):
        lam, fit, st = oracle.cp_als_iter(idx, vals, dims, A, R, xnorm2=x2)
        assert st == 0
        fits.append(fit)
        if fit > 1 - 1e-7:
            break
    assert fits[-1] > 1 - 1e-6, fits[-5:]
    # ALS never increases the residual (up to rounding)
    assert all(b >= a - 1e-10 for a, b in zip(fits, fits[1:]))


def test_cp_als_fit_and_normal_equations():
    dims = (9, 8, 7)
    R = 4
    idx, vals = synth.coo_uniform_distinct(dims, 150, 3)
    v64 = vals.astype(np.float64)
    rng = np.random.default_rng(7)
    A = [rng.uniform(0, 1, (I, R)) for I in dims]
    lam, fit, st = oracle.cp_als_iter(idx, v64, dims, A, R)
    assert st == 0
    # fit against the dense residual ||X - M|| / ||X||
    X = _dense(idx, v64, dims)
    M = np.einsum("r,ir,jr,kr->ijk", lam, *A)
    ref = 1 - np.linalg.norm(X - M) / np.linalg.norm(X)
    assert abs(fit - ref) < 1e-10
    # columns are unit norm, lambda >= 0
    for f in A:
        np.testing.assert_allclose(np.linalg.norm(f, axis=0), 1.0, rtol=1e-12)
    assert (lam >= 0).all()
    # last mode satisfies its normal equations with the final factors:
    # MTTKRP_3(X, A) = (A3 diag(lam)) (G1 * G2)
    V = oracle.mttkrp(idx, v64, dims, A, 2, R)
    H = (A[0].T @ A[0]) * (A[1].T @ A[1])
    np.testing.assert_allclose(V, (A[2] * lam[None, :]) @ H, rtol=1e-9, atol=1e-10)


def _ref_bf16(x: float) -> float:
    """bfloat16 round-to-nearest-even written on the IEEE bit fields of a
    double: keep the top k bits of the 53-bit integer significand M (k = 8 for
    normal bfloat16 results, fewer below 2^-126 where the spacing stays
    2^-133), add one to the kept part when the dropped bits exceed half of its
    last place, or equal half and the kept part is odd; overflow past the
    largest finite bfloat16, 0x7f7f = 255 * 2^120, gives infinity."""
    if x == 0.0 or not math.isfinite(x):
        return x
    bits = struct.unpack("<Q", struct.pack("<d", x))[0]
    sign = -1.0 if bits >> 63 else 1.0
    ef = (bits >> 52) & 0x7FF
    if ef == 0:  # a double subnormal: far below half the smallest bfloat16
        return sign * 0.0
    E = ef - 1023
    M = (bits & ((1 << 52) - 1)) | (1 << 52)
    k = 8 if E >= -126 else E + 134
    if k < 0:
        return sign * 0.0
    drop = 53 - k
    q, rem, half = M >> drop, M & ((1 << drop) - 1), 1 << (drop - 1)
    if rem > half or (rem == half and (q & 1)):
        q += 1
    r = math.ldexp(q, E - 52 + drop)
    if r > 255.0 * 2.0 ** 120:
        return sign * math.inf
    return sign * r


def _bf16_pin_values() -> np.ndarray:
    """Exact ties (even and odd kept parts) in several binades, their
    neighbours one double ulp away, bfloat16 subnormals with their ties, the
    underflow and overflow thresholds, signed zeros and random values."""
    v = []
    for e in (-100, -20, -1, 0, 3, 60, 127):
        for j in range(128):
            base = 1.0 + j * 2.0 ** -7
            tie = math.ldexp(base + 2.0 ** -8, e)
            v += [math.ldexp(base, e), tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf)]
    for j in range(0, 128):  # subnormal bfloat16: multiples of 2^-133
        tie = (j + 0.5) * 2.0 ** -133
        v += [j * 2.0 ** -133, tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf)]
    v += [2.0 ** -126, np.nextafter(2.0 ** -126, 0.0), 2.0 ** -134, 2.0 ** -134 * (1 + 2.0 ** -20),
          2.0 ** -135, 5e-324, 255.0 * 2.0 ** 120, 255.5 * 2.0 ** 120,
          np.nextafter(255.5 * 2.0 ** 120, 0.0), 2.0 ** 128, 1e300, 0.0, -0.0]
    rng = np.random.default_rng(7)
    v += list(rng.uniform(0.0, 1.0, 3000))
    v += list(np.exp(rng.uniform(-300.0, 90.0, 3000)) * rng.choice([-1.0, 1.0], 3000))
    a = np.array(v, dtype=np.float64)
    return np.concatenate([a, -a])


def test_round_bf16_is_bitwise_round_to_nearest_even():
    x = _bf16_pin_values()
    got = oracle.round_bf16(x)
    ref = np.array([_ref_bf16(float(t)) for t in x])
    bad = np.nonzero(got.view(np.uint64) != ref.view(np.uint64))[0]
    assert bad.size == 0, [(x[i], got[i], ref[i]) for i in bad[:5]]


def test_round_bf16_agrees_with_torch_on_float32_inputs():
    # torch's CPU float32 -> bfloat16 conversion (round to nearest even) on
    # values that are exactly float32, including float32 subnormals
    import torch
    v = _bf16_pin_values()
    x = v[np.abs(v) < 3.0e38].astype(np.float32).astype(np.float64)
    got = oracle.round_bf16(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_cp_als_bf16_rounding_keeps_values_on_bf16_grid():
    dims = (9, 8, 7)
    R = 4
    idx, vals = synth.coo_uniform_distinct(dims, 150, 4)
    rng = np.random.default_rng(8)
    A = [rng.uniform(0, 1, (I, R)) for I in dims]
    oracle.cp_als_iter(idx, vals, dims, A, R, bf16=True)
    import torch
    for f in A:
        t = torch.from_numpy(f.astype(np.float32))
        back = t.to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(back, f)  # already representable in bf16


def test_cp_als_singular_gram_reports_status():
    dims = (6, 5, 4)
    R = 3
    idx, vals = synth.coo_uniform_distinct(dims, 30, 2)
    # identical columns give rank-1 Grams: the ridge retry rescues the solve
    A = [np.ones((I, R)) for I in dims]
    _, _, st = oracle.cp_als_iter(idx, vals, dims, A, R)
    assert st == 0
    # all-zero factors give H = 0, which no ridge proportional to trace(H) fixes
    A = [np.zeros((I, R)) for I in dims]
    _, _, st = oracle.cp_als_iter(idx, vals, dims, A, R)
    assert st == 2


def _mlp_params(F, H1, H2, K, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((H1, F)) * 0.5, rng.standard_normal(H1) * 0.1,
            rng.standard_normal((H2, H1)) * 0.3, rng.standard_normal(H2) * 0.1,
            rng.standard_normal((K, H2)) * 0.3, rng.standard_normal(K) * 0.1]


def test_mlp_forward_matches_matrix_products():
    F, H1, H2, K, B = 7, 9, 8, 5, 6
    p = _mlp_params(F, H1, H2, K, 0)
    X = np.random.default_rng(1).standard_normal((B, F))
    relu = lambda z: np.maximum(z, 0)
    ref = relu(relu(X @ p[0].T + p[1]) @ p[2].T + p[3]) @ p[4].T + p[5]
    np.testing.assert_allclose(oracle.mlp_forward(X, p), ref, rtol=1e-13, atol=1e-13)


def test_mlp_gradient_matches_finite_differences():
    F, H1, H2, K, B = 5, 6, 7, 4, 8
    p = _mlp_params(F, H1, H2, K, 2)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((B, F))
    T = rng.standard_normal((B, K))
    M = (rng.random((B, K)) < 0.7).astype(np.float64)
    loss, grads = oracle.mlp_loss_grad(X, p, T, M)
    h = 1e-6
    for pi, (P_, G_) in enumerate(zip(p, grads)):
        flat = P_.reshape(-1)
        gflat = G_.reshape(-1)
        for q in range(flat.size):
            old = flat[q]
            flat[q] = old + h
            lp, _ = oracle.mlp_loss_grad(X, p, T, M)
            flat[q] = old - h
            lm, _ = oracle.mlp_loss_grad(X, p, T, M)
            flat[q] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[q]) <= 1e-6 * max(1.0, abs(fd)), (pi, q, fd, gflat[q])


# ---- generalised CP gradient: pinned by the dense loss and its finite differences

def _dense_model(factors):
    d = len(factors)
    letters = "abcdefg"[:d]
    return np.einsum(",".join(f"{c}r" for c in letters) + "->" + letters, *factors)


def _gcp_loss_dense(idx, vals, dims, factors, loss):
    """F from the dense model tensor M: Poisson over every entry of the dense
    tensor (duplicates summed), the other losses over the stored list."""
    M = _dense_model(factors)
    if loss == "poisson":
        X = _dense(idx, vals, dims)
        return float(M.sum() - (X[X > 0] * np.log(M[X > 0])).sum())
    m = M[tuple(idx.astype(np.int64))]
    x = vals.astype(np.float64)
    if loss == "bernoulli":
        return float((np.logaddexp(0.0, m) - x * m).sum())
    return float(((m - x) ** 2).sum())


@pytest.mark.parametrize("loss", ["poisson", "bernoulli", "gaussian"])
@pytest.mark.parametrize("d", [3, 4])
def test_gcp_gradient_is_the_derivative_of_the_dense_loss(loss, d):
    dims = (5, 4, 3, 3)[:d]
    R = 3
    idx, vals = synth.coo_zipf(dims, 40, 0.7, 3 + d)  # duplicates included
    if loss == "bernoulli":
        vals = (vals > 0.5).astype(np.float32)
    rng = np.random.default_rng(d)
    A = [rng.random((I, R)) + 0.2 for I in dims]
    for n in range(d):
        G, F = oracle.gcp_grad(idx, vals, dims, A, n, R, loss)
        assert abs(F - _gcp_loss_dense(idx, vals, dims, A, loss)) <= 1e-10 * max(1.0, abs(F))
        h = 1e-6
        fd = np.zeros_like(G)
        for k in range(dims[n]):
            for j in range(R):
                Ap = [a.copy() for a in A]
                Am = [a.copy() for a in A]
                Ap[n][k, j] += h
                Am[n][k, j] -= h
                fd[k, j] = (_gcp_loss_dense(idx, vals, dims, Ap, loss) -
                            _gcp_loss_dense(idx, vals, dims, Am, loss)) / (2 * h)
        assert np.abs(G - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max()), (loss, n)


def test_gcp_gaussian_on_a_full_tensor_is_the_normal_equation_residual():
    """With every coordinate stored once, the Gaussian gradient is
    2 (A^(n) *_{l != n} A^(l)T A^(l) - MTTKRP_n(X)): the CP-ALS normal equation."""
    dims = (4, 3, 5)
    R = 2
    idx = np.array(list(itertools.product(*[range(I) for I in dims]))).T.astype(np.int32)
    vals = np.random.default_rng(0).random(idx.shape[1]).astype(np.float32)
    rng = np.random.default_rng(1)
    A = [rng.standard_normal((I, R)) for I in dims]
    for n in range(3):
        G, _ = oracle.gcp_grad(idx, vals, dims, A, n, R, "gaussian")
        H = np.ones((R, R))
        for l in range(3):
            if l != n:
                H *= A[l].T @ A[l]
        V = oracle.mttkrp(idx, vals, dims, A, n, R)
        np.testing.assert_allclose(G, 2 * (A[n] @ H - V), rtol=1e-10, atol=1e-10)

"""gloo tests of the nonzero-sharded CP-ALS on two and three ranks (CPU only).

The distribution of ``paper_1809_09175_gb300.shard`` -- every rank holds a
contiguous range of each mode's permutation and owns the rows it reaches
first, the rows shared at the cuts completed by one small all-reduce, the
owned rows solved, the column norms and the R x R Grams all-reduced, each
rank's factor rows broadcast -- runs here on gloo ranks, including a case
whose hot rows span whole ranks (ranks that own no row of a mode).
The rank-local steps that run in CUDA kernels on a GPU are done in FP64 on
the host: the MTTKRP of the rank's nonzeros by the oracle, the small dense
steps by numpy.  One sharded iteration must then reproduce the oracle's
single-process CP-ALS iteration element by element.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(name):
    import synth
    if name == "zipf3":
        dims, R = (41, 37, 29), 5
        idx, vals = synth.coo_zipf(dims, 3000, 0.9, 17)
    elif name == "zipf4_short_mode":  # a 4-way tensor with a 3-row mode
        dims, R = (23, 3, 19, 11), 4
        idx, vals = synth.coo_zipf(dims, 1500, 0.6, 18)
    else:  # mode-0 row 7 holds 1200 of 1500 draws (about 3/4 of the coalesced
        # nonzeros), so on three ranks the middle rank's range lies inside it
        # and that rank owns no row of mode 0
        dims, R = (30, 40, 35), 4
        rng = np.random.default_rng(19)
        idx = np.stack([np.where(np.arange(1500) < 1200, 7, rng.integers(0, dims[0], 1500)),
                        rng.integers(0, dims[1], 1500), rng.integers(0, dims[2], 1500)]).astype(np.int32)
        vals = rng.random(1500).astype(np.float32)
    import oracle
    idx, vals = oracle.coalesce(idx, vals)
    return dims, R, idx, vals.astype(np.float64)


class HostOps:
    """The rank-local steps in FP64 on the host (the oracle's MTTKRP and
    numpy's dense algebra), standing in for the CUDA kernels."""

    acc_dtype = torch.float64

    def __init__(self, dims, R, shards):
        self.dims, self.R, self.shards = dims, R, shards

    def row_span(self, mode):
        idx, _ = self.shards[mode]
        if idx.shape[1] == 0:
            return -1, -1
        return int(idx[mode, 0]), int(idx[mode, -1])

    def partial_mttkrp(self, mode, factors, V):
        import oracle
        idx, vals = self.shards[mode]
        V.zero_()
        A = [f[:, : self.R].numpy() for f in factors]
        V[: self.dims[mode], : self.R] = torch.from_numpy(oracle.mttkrp(idx, vals, self.dims, A, mode, self.R))

    def gram(self, A, rows, G):
        a = A[:rows, : self.R]
        G.copy_(a.T @ a)

    def solve_rows(self, mode, Grams, Vr, rows, A32, colsq):
        H = torch.ones((self.R, self.R), dtype=torch.float64)
        for m in range(len(self.dims)):
            if m != mode:
                H = H * Grams[m]
        A32.zero_()
        A32[:rows, : self.R] = torch.linalg.solve(H, Vr[:rows, : self.R].T).T
        colsq.copy_((A32[:rows, : self.R] ** 2).sum(0))

    def normalize_rows(self, A32, rows, colsq, Ar, lam, Vr, inner):
        lam.copy_(torch.sqrt(colsq))
        scale = torch.where(lam > 0, lam, torch.ones_like(lam))
        Ar.zero_()
        Ar[:rows, : self.R] = A32[:rows, : self.R] / scale
        if inner is not None:
            inner[0] = (Vr[:rows, : self.R] * lam * Ar[:rows, : self.R]).sum()

    def fit(self, Grams, lam, inner, x2, fit):
        H = torch.ones((self.R, self.R), dtype=torch.float64)
        for m in range(len(self.dims)):
            H = H * Grams[m]
        m2 = float(lam @ H @ lam)
        fit[0] = 1.0 - np.sqrt(max(0.0, x2 + m2 - 2.0 * float(inner[0]))) / np.sqrt(x2)

    def check(self):
        pass

    def xnorm2(self):
        return float((self.shards[0][1] ** 2).sum())


def _worker(rank, world, port, out_dir, name):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1809_09175_gb300 import shard as S

    dims, R, idx, vals = _case(name)
    shards = []
    for n in range(len(dims)):  # this rank's contiguous range of perm_n
        perm = oracle.stable_argsort(idx[n])
        b, e = S.shard_bounds(idx.shape[1], world, rank)
        sel = perm[b:e]
        shards.append((idx[:, sel], vals[sel]))
    ld = synth.padded_ld(R)
    facs = [torch.from_numpy(f.astype(np.float64)) for f in synth.factor_matrices(dims, R, 5, "uniform")]
    drv = S.ShardedCPALS(HostOps(dims, R, shards), dims, R, ld)
    F = drv.replicated_factors(facs)
    lam = torch.zeros(R, dtype=torch.float64)
    fit = torch.zeros(1, dtype=torch.float64)
    drv.step(F, lam, fit)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), lam=lam.numpy(), fit=fit.numpy(),
             **{f"A{m}": F[m][:, :R].numpy() for m in range(len(dims))},
             **{f"P{m}": F[m][:, R:].numpy() for m in range(len(dims))},
             own=np.array([[lo, hi] for n in range(len(dims)) for lo, hi in drv.own[n]]))
    dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("zipf3", 2), ("zipf4_short_mode", 2), ("hot_rows", 3)])
def test_gloo_ranks_match_one_oracle_iteration(tmp_path, name, world):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), name), nprocs=world, join=True)
    dims, R, idx, vals = _case(name)
    A = [f[:, :R].astype(np.float64).copy() for f in synth.factor_matrices(dims, R, 5, "uniform")]
    lam_o, fit_o, st = oracle.cp_als_iter(idx, vals, dims, A, R)
    assert st == 0
    for r in range(world):
        z = np.load(tmp_path / f"r{r}.npz")
        for m in range(len(dims)):  # replicated factors, equal to the oracle's
            np.testing.assert_allclose(z[f"A{m}"], A[m], rtol=1e-10, atol=1e-12)
            assert not z[f"P{m}"].any()  # the padding columns stay zero
        np.testing.assert_allclose(z["lam"], lam_o, rtol=1e-10)
        assert abs(float(z["fit"][0]) - fit_o) <= 1e-10
    if name == "hot_rows":  # the middle rank owns no row of mode 0
        own = np.load(tmp_path / "r0.npz")["own"]
        assert own[1][0] == own[1][1] and own[0][1] > 7 and own[0][0] <= 7


def test_shard_bounds_and_owned_rows_partition():
    import sys
    sys.path.insert(0, ROOT)
    from paper_1809_09175_gb300 import shard as S
    for P_, G in [(0, 3), (1, 4), (10, 3), (1001, 8)]:
        b = [S.shard_bounds(P_, G, r) for r in range(G)]
        assert b[0][0] == 0 and b[-1][1] == P_
        assert all(b[r][1] == b[r + 1][0] for r in range(G - 1))
        assert max(e - s for s, e in b) - min(e - s for s, e in b) <= 1
    # last rows per rank (-1: no nonzeros) -> owned [lo, hi): consecutive,
    # covering [0, I), every last row owned by the first rank reaching it
    cases = [([4, 9], 12), ([-1, 3, 3, 7], 8), ([5, 5, 5], 6), ([-1, -1, 0], 1), ([2, 2, -1], 10)]
    for lasts, I in cases:
        own = S.owned_rows(lasts, I)
        assert own[0][0] == 0 and own[-1][1] == I
        assert all(own[r][1] == own[r + 1][0] for r in range(len(own) - 1))
        for r, L in enumerate(lasts):
            if L >= 0:
                first_reach = min(q for q in range(len(lasts)) if lasts[q] >= L)
                assert S.row_owner(own, L) == first_reach
    assert S.owned_rows([5, 5, 5], 6) == [(0, 6), (6, 6), (6, 6)]
    assert S.owned_rows([-1, 3, 3, 7], 8) == [(0, 0), (0, 4), (4, 4), (4, 8)]
    with pytest.raises(ValueError):
        S.row_owner([(0, 2), (2, 2)], 2)

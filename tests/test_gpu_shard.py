"""GPU tests of the nonzero-sharded CP-ALS pieces: tensor_create_shard and
the per-step C ABI (cp_als_hinv / _apply / _normalize / _gram / _fit) driven
by paper_1809_09175_gb300.shard over a one-rank NCCL group (this machine has
one GPU; the two-rank distribution is covered by the gloo tests on CPU)."""
import os
import socket

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


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.fixture
def nccl_one_rank():
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    yield
    dist.destroy_process_group()


def test_shards_cover_the_permutation_in_order():
    P = _lib()
    dims = (700, 500, 300)
    idx, vals = synth.coo_zipf(dims, 50_000, 1.0, 9)
    T = P.SparseTensor(idx, vals, dims, coalesce=True)
    T.build_permutation()
    c_idx, c_vals = (a.cpu().numpy() for a in T.coo())
    for n in range(3):
        perm = oracle.stable_argsort(c_idx[n])
        total = 0.0
        for r in range(3):
            b, e = P.shard.shard_bounds(T.nnz, 3, r)
            S = P.SparseTensor.from_handle(P.tensor_create_shard(T.handle, n, b, e), dims)
            s_idx, s_vals = (a.cpu().numpy() for a in S.coo())
            np.testing.assert_array_equal(s_idx, c_idx[:, perm[b:e]])
            np.testing.assert_array_equal(s_vals, c_vals[perm[b:e]])
            assert S.coalesced
            total += S.norm2()
            S.close()
        assert abs(total - T.norm2()) <= 1e-9 * T.norm2()
    with pytest.raises(P.SptError):
        P.tensor_create_shard(T.handle, 0, 10, 5)
    T.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_one_rank_sharded_iteration_matches_oracle_and_cp_als_step(nccl_one_rank, dtype):
    P = _lib()
    from paper_1809_09175_gb300 import shard as S
    from tests.test_gpu_cpals import U32, _gram_hadamard_conds
    dims = (2000, 1500, 1000)
    R = 16
    idx, vals = synth.coo_zipf(dims, 200_000, 1.0, 4)
    T = P.SparseTensor(idx, vals, dims, coalesce=True)
    T.build_permutation()
    shards = S.make_shards(T, 1, 0)
    facs_np = synth.factor_matrices(dims, R, 4, "uniform", dtype=dtype)
    facs = [to_device_factor(f, dtype) for f in facs_np]
    ld = facs[0].shape[1]
    drv = S.ShardedCPALS(S.DeviceOps(T, shards, R, dtype, ld), dims, R, ld)
    F = drv.replicated_factors(facs)
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    drv.step(F, lam, fit)
    torch.cuda.synchronize()
    # the oracle's iteration from the same stored values on the coalesced nonzeros
    c_idx, c_vals = (a.cpu().numpy() for a in T.coo())
    A = [oracle.as_f64(f, dtype)[:, :R].copy() for f in facs_np]
    A_old = [a.copy() for a in A]
    lam_o, fit_o, st = oracle.cp_als_iter(c_idx, c_vals, dims, A, R, bf16=(dtype == "bf16"))
    assert st == 0
    if dtype == "f32":
        tols = [max(1e-5, 4.0 * c * U32) for c in _gram_hadamard_conds(A_old, A)]
    else:
        tols = [2e-3] * 3
    for m in range(3):
        got = F[m][: dims[m], :R].float().cpu().numpy().astype(np.float64)
        assert rel_fro(got, A[m]) <= tols[m], (m, rel_fro(got, A[m]), tols[m])
    assert rel_fro(lam.cpu().numpy(), lam_o) <= tols[-1]
    assert abs(float(fit.item()) - fit_o) <= tols[-1]
    # the single-GPU cp_als_step from the same factors takes the same kernels
    g = [to_device_factor(f, dtype) for f in facs_np]
    lam2 = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = T.cp_als_workspace(R, ld)
    T.cp_als_step(g, R, lam2, fit2, ws)
    torch.cuda.synchronize()
    assert abs(float(fit2.item()) - float(fit.item())) <= tols[-1]
    for s_ in shards:
        s_.close()
    T.close()


def test_phase_calls_check_their_arguments():
    P = _lib()
    with pytest.raises(P.SptError) as e:
        P.cp_als_hinv(0, 3, 0, 16, 0, 0)
    assert e.value.status == P.SPT_EINVAL
    G = torch.zeros((3, 16, 16), dtype=torch.float64, device="cuda")
    h = torch.zeros((16, 16), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(P.SptError) as e:
        P.cp_als_hinv(G.data_ptr(), 3, 3, 16, h.data_ptr(), st.data_ptr())
    assert e.value.status == P.SPT_EINVAL
    with pytest.raises(P.SptError) as e:
        P.cp_als_gram(G.data_ptr(), 4, 12, 16, "f32", G.data_ptr())  # ld < rank
    assert e.value.status == P.SPT_EINVAL
    # a singular H (zero Grams) is reported through the status word
    P.cp_als_hinv(G.data_ptr(), 3, 0, 16, h.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    assert int(st.item()) == 2

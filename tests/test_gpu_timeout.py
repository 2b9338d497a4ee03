"""GPU tests of the failure-detection path: a bounded device wait that runs out.

Every staging wait of the MTTKRP kernels is bounded.  spt_set_wait_tries(0)
makes each such wait give up at once, without looking, so the timeout path
runs on a healthy GPU with no fault: the warp records SPT_DEV_TIMEOUT in the
status word, lets its own bulk copies land (with the full default budget),
and returns.  The host must then see SPT_ETIMEOUT, and a normal call after
the budget is restored must succeed and be correct.
"""
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


def _case():
    dims = (300, 200, 100)
    idx, vals = synth.coo_zipf(dims, 20_000, 0.9, 11)
    R = 16
    facs_np = synth.factor_matrices(dims, R, 11, "uniform")
    return dims, idx, vals, R, facs_np


@pytest.mark.parametrize("scatter", ["sorted", "atomic", "perm", "private", "deterministic"])
def test_expired_wait_is_reported_and_the_next_call_recovers(scatter):
    P = _lib()
    dims, idx, vals, R, facs_np = _case()
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    facs = [to_device_factor(f, "f32") for f in facs_np]
    det = scatter == "deterministic"
    sched = P.spt_schedule.make("sorted" if det else scatter, lanes_per_nnz=4, chunks=1, nnz_per_group=15,
                                warps_per_cta=4)
    try:
        P.spt_set_wait_tries(0)
        T.mttkrp(0, facs, R, sched=sched, deterministic=det)
        with pytest.raises(P.SptError) as e:
            T.check()
        assert e.value.status == P.SPT_ETIMEOUT
    finally:
        P.spt_set_wait_tries(-1)
    T.check()  # the reported status was cleared
    ref = oracle.mttkrp(idx, vals, dims, [widen(f, "f32", R) for f in facs_np], 0, R)
    got = T.mttkrp(0, facs, R, sched=sched, deterministic=det)
    T.check()
    assert rel_fro(got.cpu().numpy()[:, :R], ref) <= 1e-5
    T.close()


def test_expired_wait_in_a_batch_is_reported():
    P = _lib()
    dims, idx, vals, R, facs_np = _case()
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    facs = [to_device_factor(f, "f32") for f in facs_np]
    outs = [torch.zeros((I, facs[0].shape[1]), device="cuda") for I in dims]
    item = {"tensor": T.handle, "mode": -1, "rank": R, "ld": facs[0].shape[1],
            "factors": [f.data_ptr() for f in facs], "outs": [o.data_ptr() for o in outs]}
    try:
        P.spt_set_wait_tries(0)  # the batch's task table takes the budget at creation
        b, keep = P.mttkrp_batch_create([item], "f32")
    finally:
        P.spt_set_wait_tries(-1)
    P.mttkrp_batch_run(b)  # legacy default stream: launched directly
    with pytest.raises(P.SptError) as e:
        P.mttkrp_batch_check(b)
    assert e.value.status == P.SPT_ETIMEOUT
    P.mttkrp_batch_check(b)  # cleared
    P.mttkrp_batch_destroy(b)
    b, keep = P.mttkrp_batch_create([item], "f32")  # default budget
    P.mttkrp_batch_run(b)
    P.mttkrp_batch_check(b)
    for n in range(3):
        ref = oracle.mttkrp(idx, vals, dims, [widen(f, "f32", R) for f in facs_np], n, R)
        assert rel_fro(outs[n].cpu().numpy()[:, :R], ref) <= 1e-5
    P.mttkrp_batch_destroy(b)
    T.close()


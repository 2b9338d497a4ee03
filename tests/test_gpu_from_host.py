"""GPU: MTTKRP from host memory (mttkrp_from_host).  The results match the
FP64 oracle and the device-pointer entry point; listed subsets of modes in
any order, pinned and pageable host buffers, fp32 / bf16 / fp64 factors;
back-to-back calls that reuse one workspace without a host synchronisation
in between keep their inputs and outputs apart; integer cases are exact;
bad arguments return statuses."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import TOL, rel_fro, widen

pytestmark = pytest.mark.gpu

def _lib():
    import paper_1809_09175_gb300 as P
    return P


def _host(f, dtype, pin=True):
    f = np.ascontiguousarray(f)
    t = torch.from_numpy(f.view(np.int16)).view(torch.bfloat16) if dtype == "bf16" else torch.from_numpy(f)
    return t.pin_memory() if pin else t


def _oracle(idx, vals, dims, facs, dtype, R, n):
    return oracle.mttkrp(idx, vals, dims, [widen(f, dtype, R) for f in facs], n, R)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("order,R,modes", [(3, 16, [0, 1, 2]), (4, 20, [2, 0, 3, 1]), (3, 40, [1]),
                                           (5, 8, [4, 3])])
def test_from_host_matches_oracle_and_device_entry(order, R, modes, dtype):
    P = _lib()
    dims = [900, 700, 300, 40, 9][:order]
    idx, vals = synth.coo_zipf(dims, 90_001, 1.2, 70 + order)
    facs = synth.factor_matrices(dims, R, 5, "uniform", dtype=dtype)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    needed = {m for n in modes for m in range(order) if m != n}
    hf = [_host(f, dtype) if m in needed else None for m, f in enumerate(facs)]
    outs = T.mttkrp_from_host(modes, hf, R)
    dev = [h.cuda() if h is not None else None for h in hf]
    for q, n in enumerate(modes):
        got = outs[q].numpy()
        assert got.shape == (dims[n], facs[0].shape[1])
        assert np.all(got[:, R:] == 0)
        assert rel_fro(got[:, :R], _oracle(idx, vals, dims, facs, dtype, R, n)) <= TOL[dtype]
        ref = T.mttkrp(n, dev, R).cpu().numpy()
        assert rel_fro(got, ref) <= (1e-13 if dtype == "f64" else 1e-6)
    T.check()
    T.close()


def test_from_host_pageable_buffers_and_integer_case():
    P = _lib()
    dims = (300, 200, 50, 7)
    R = 13
    idx, vals, facs = synth.small_integer_case(dims, 40_000, R, 5)
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    hf = [_host(f, "f32", pin=False) for f in facs]
    outs = [torch.empty((I, facs[0].shape[1]), dtype=torch.float32) for I in dims]  # pageable
    T.mttkrp_from_host([3, 2, 1, 0], hf, R, outs=[outs[3], outs[2], outs[1], outs[0]])
    for n in range(4):
        ref = _oracle(idx, vals, dims, facs, "f32", R, n)
        np.testing.assert_array_equal(outs[n].numpy()[:, :R], ref.astype(np.float32))
    T.close()


def test_from_host_back_to_back_calls_share_the_workspace():
    """Two calls queued without a host synchronisation, different factors and
    outputs, one workspace: the second call's uploads must wait for the first
    call's kernels, and its kernels for the first call's downloads."""
    P = _lib()
    dims = (2000, 1500, 800)
    R = 16
    idx, vals = synth.coo_zipf(dims, 400_003, 1.1, 3)
    fa = synth.factor_matrices(dims, R, 11, "normal")
    fb = synth.factor_matrices(dims, R, 12, "normal")
    T = P.SparseTensor(idx, vals, dims)
    T.build_permutation()
    ld = fa[0].shape[1]
    ws = torch.empty(P.mttkrp_from_host_workspace_size(T.handle, [0, 1, 2], "f32", R, ld),
                     dtype=torch.uint8, device="cuda")
    oa = T.mttkrp_from_host([0, 1, 2], [_host(f, "f32") for f in fa], R, workspace=ws, sync=False)
    ob = T.mttkrp_from_host([0, 1, 2], [_host(f, "f32") for f in fb], R, workspace=ws, sync=False)
    torch.cuda.synchronize()
    for facs, outs in ((fa, oa), (fb, ob)):
        for n in range(3):
            ref = _oracle(idx, vals, dims, facs, "f32", R, n)
            assert rel_fro(outs[n].numpy()[:, :R], ref) <= TOL["f32"], n
    T.close()


def test_from_host_errors():
    P = _lib()
    dims = (30, 20, 10)
    R = 8
    idx, vals = synth.coo_zipf(dims, 500, 0.5, 1)
    T = P.SparseTensor(idx, vals, dims)
    hf = [torch.rand((I, R)).pin_memory() for I in dims]
    need = P.mttkrp_from_host_workspace_size(T.handle, [0, 1], "f32", R, R)
    assert need % 256 == 0 and need >= (30 + 20 + 10 + 30 + 20) * R * 4
    with pytest.raises(P.SptError) as ei:  # a repeated mode
        T.mttkrp_from_host([0, 0], hf, R)
    assert ei.value.status == P.SPT_EINVAL
    with pytest.raises(P.SptError) as ei:  # a factor mode 0 reads is missing
        T.mttkrp_from_host([0], [hf[0], None, hf[2]], R)
    assert ei.value.status == P.SPT_EINVAL
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    outs = [torch.empty((I, R)).pin_memory() for I in dims[:2]]
    with pytest.raises(P.SptError) as ei:
        P.mttkrp_from_host(T.handle, [0, 1], [h.data_ptr() for h in hf], "f32", R, R, 0,
                           [o.data_ptr() for o in outs], small.data_ptr(), small.numel(),
                           torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == P.SPT_EINVAL
    out = T.mttkrp_from_host([1], [hf[0], None, hf[2]], R)[0]  # factors[1] is not read
    ref = oracle.mttkrp(idx, vals, dims, [h.numpy().astype(np.float64) for h in hf], 1, R)
    assert rel_fro(out.numpy(), ref) <= TOL["f32"]
    T.close()

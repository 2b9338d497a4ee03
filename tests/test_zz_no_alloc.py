"""The allocation-free mode permutation against build_mode_permutation.

mode_permutation_noalloc serves callers that cannot allocate device memory
when they sort (a process whose memory pool owns the whole GPU, or code that
must avoid the device-wide synchronisation of cudaFree): it sorts inside a
static scratch array that ships with the library.  Its result must be the
same permutation build_mode_permutation produces, call after call, even
though every call reuses the same scratch array.  This file is collected
last so a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _reference_perm(P, keys_np, dim):
    """perm_n from the allocating entry point (a one-mode tensor)."""
    T = P.SparseTensor(keys_np[None, :], np.ones(keys_np.shape[0], np.float32), (dim,))
    T.build_permutation(0, index_only=True)
    out = T.permutation(0).cpu().numpy()
    T.close()
    return out


def test_noalloc_permutation_matches_allocating_entry_point_twice():
    import paper_1809_09175_gb300 as P
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    cases = [(1_000_003, 300_000), (P.SPT_NOALLOC_MAX_NNZ, 2_000_000)]
    for n, dim in cases:  # two calls in a row through the same scratch array
        keys_np = rng.integers(0, dim, n).astype(np.int32)
        keys_np[: n // 7] = dim // 3  # a hot coordinate: long runs of equal keys
        keys = torch.from_numpy(keys_np).cuda()
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        P.mode_permutation_noalloc(keys.data_ptr(), n, dim, perm.data_ptr(), stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(perm.cpu().numpy(), _reference_perm(P, keys_np, dim))


@pytest.mark.parametrize("n,dim", [(5000, 1), (70_001, 200), (1, 256), (300_000, 257), (123_457, 65_536)])
def test_noalloc_one_and_two_pass_sorts_match(n, dim):
    """Key ranges of one 8-bit digit (one pass, keys straight to perm), two
    digits (two passes), and a single coordinate value (dim = 1)."""
    import paper_1809_09175_gb300 as P
    stream = torch.cuda.current_stream().cuda_stream
    keys_np = np.random.default_rng(n + dim).integers(0, dim, n).astype(np.int32)
    keys = torch.from_numpy(keys_np).cuda()
    ref = _reference_perm(P, keys_np, dim)
    for _ in range(2):  # the second call starts from the first call's scratch contents
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        P.mode_permutation_noalloc(keys.data_ptr(), n, dim, perm.data_ptr(), stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(perm.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_the_scratch_area():
    import paper_1809_09175_gb300 as P
    keys = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(P.SptError) as ei:
        P.mode_permutation_noalloc(keys.data_ptr(), P.SPT_NOALLOC_MAX_NNZ + 1, 10, keys.data_ptr())
    assert ei.value.status == P.SPT_EINVAL
    assert "static scratch" in P.spt_last_error()

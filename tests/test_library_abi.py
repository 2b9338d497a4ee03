"""The compiled library loads without a GPU and exports every entry point
that include/spt.h declares; argument checks that need no device memory
return their status codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    import paper_1809_09175_gb300 as P
    L = P.binding.lib()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    import paper_1809_09175_gb300 as P
    missing = [n for n in _declared() if n not in P.binding.EXPORTED]
    assert not missing, missing


def test_argument_errors_without_device():
    import paper_1809_09175_gb300 as P
    with pytest.raises(P.SptError) as ei:
        P.tensor_create_coo(0, [], 0, [], 0)
    assert ei.value.status == P.SPT_EINVAL
    with pytest.raises(P.SptError) as ei:
        P.tensor_create_coo(3, [4, 0, 2], 0, [0, 0, 0], 0)
    assert ei.value.status == P.SPT_EINVAL
    with pytest.raises(P.SptError) as ei:
        P.tensor_create_coo(2, [4, 4], 5, [0, 0], 0)
    assert ei.value.status == P.SPT_EINVAL
    assert "NULL" in P.spt_last_error()
    L = P.binding.lib()  # NULL tensors: refused before any device work
    n = C.c_size_t()
    modes = (C.c_int * 1)(0)
    assert L.mttkrp_from_host_workspace_size(None, 1, modes, 0, 8, 8, C.byref(n)) == P.SPT_EINVAL
    assert L.mttkrp_from_host(None, 1, modes, None, 0, 8, 8, None, None, None, 0, None) == P.SPT_EINVAL
    assert L.mttkrp_deterministic(None, 0, None, 0, 8, 8, None, None, None, None) == P.SPT_EINVAL
    assert L.gcp_gradient(None, 0, None, 0, 8, 8, 0, None, None, None) == P.SPT_EINVAL
    assert L.build_mode_l2_blocks(None, 0, -1, -1, None) == P.SPT_EINVAL
    assert L.tensor_storage_records(None, 1, None) == P.SPT_EINVAL
    assert L.tensor_l2_blocks(None, 0, None, None, None) == P.SPT_EINVAL
    for bad in (-2, 1 << 32):  # the wait budget is host state: checked without a device
        with pytest.raises(P.SptError) as ei:
            P.spt_set_wait_tries(bad)
        assert ei.value.status == P.SPT_EINVAL
    P.spt_set_wait_tries(123)
    P.spt_set_wait_tries(-1)


def test_product_path_never_uses_the_oracle():
    """The package and the CUDA sources neither import, include nor load
    anything under oracle/ (the oracle is test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1809_09175_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if not fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                continue
            src = open(os.path.join(dirpath, fn)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), fn
            assert "liboracle" not in src and "oracle.c" not in src and "oracle/" not in src, fn
            assert not re.search(r'#include\s+"[^"]*oracle', src), fn


def test_paper_sizes_table_matches_golden():
    """Tab. "sizes" (Sec. 5) as printed: vector_size and FBS for each R range."""
    import paper_1809_09175_gb300 as P
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_tab_sizes.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append([int(x) for x in line.split()])
    assert len(rows) == 13
    for lo, hi, vs, fbs in rows:
        for R in sorted({lo, hi, (lo + hi) // 2}):
            assert P.mttkrp_paper_sizes(R) == (vs, fbs), R
    # the schedule built from the table covers FBS columns with 16-byte chunks
    for R in (1, 16, 24, 48, 64, 96, 128, 200):
        vs, fbs = P.mttkrp_paper_sizes(R)
        for fdt, vec in (("f32", 4), ("bf16", 4)):
            s = P.mttkrp_paper_schedule(R, fdt, "sorted")
            cover = s.lanes_per_nnz * s.chunks * vec
            assert cover >= fbs and s.nnz_per_group == 128 and s.warps_per_cta == 4

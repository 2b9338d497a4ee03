"""CPU checks of bench.py's host logic: the algorithmic-bytes model against
the byte counts worked out by hand for the benchmark workloads, the paper's
bandwidth model, and the reference arm's JSON line (it times the oracle on
the host, so it runs here)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("scatter,d,R,s_f,per_nnz", [
    # value 4 + d ordinals 4 + (d-1) rows of R factors (+4 through perm_n, +4R atomic)
    ("atomic", 3, 16, 4, 208), ("sorted", 3, 16, 4, 144), ("perm", 3, 16, 4, 148),
    ("sorted", 3, 16, 2, 80), ("perm", 4, 64, 4, 792), ("atomic", 4, 64, 2, 660),
    ("perm", 4, 64, 2, 408), ("perm", 5, 32, 2, 284), ("atomic", 5, 32, 2, 408),
])
def test_algorithmic_bytes_per_nonzero(scatter, d, R, s_f, per_nnz):
    b = _bench()
    P, I_n = 1000, 10
    got = b.algorithmic_bytes(scatter, P, d, R, s_f, I_n, I_n)
    out = I_n * R * 4 + (0 if scatter == "atomic" else I_n * R * 4)
    assert got == P * per_nnz + out


def test_compulsory_bytes_counts_every_input_once():
    b = _bench()
    dims = [7, 5, 3]
    # 1000 nonzeros x (value + 3 ordinals) + factor rows of the other modes + the output
    assert b.compulsory_bytes(1000, 3, dims, 0, 16, 4) == 1000 * 16 + (5 + 3) * 16 * 4 + 7 * 16 * 4


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--scale", "0.001", "--steps", "1", "--warmup", "1", "--cpu-sample", "20000"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in j, k
    assert j["impl"] == "reference" and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["e2e"]["h2d_bytes_per_step"] == 0


def test_dram_traffic_record_matches_the_kernel_sources():
    """The bench's roofline fraction divides the ncu-measured DRAM bytes of
    the committed record by the kernel time; the record must have been taken
    from the kernel sources as they are (their hash), else the bench reports
    no traffic.  A change to the kernel sources needs a new capture."""
    b = _bench().kernel_traffic(100_000_000)
    assert b is not None
    assert 16e8 <= b <= 40e8  # the 16-byte record stream plus factor-row misses, per 1e8 nonzeros

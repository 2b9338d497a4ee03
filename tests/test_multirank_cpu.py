"""World-size-2 gloo tests of the multi-rank host path (CPU only).

Each rank takes its share of a batch of tensors, computes their MTTKRPs with
the FP64 oracle (standing in for its GPU), and the job's results and timing
reductions are checked against a single-process run: sharding loses or
duplicates no work and the throughput is all units over the slowest rank.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1809_09175_gb300 import multi  # noqa: E402  (host logic only)

    specs = synth.batched_specs(6, seed0=300, nnz_scale=0.002)
    mine = multi.shard(list(enumerate(specs)), rank, world)
    units = 0.0
    for i, w in mine:
        idx, vals = w.coo()
        facs = [f[:, :w.R].astype(np.float64) for f in w.factors()]
        res = [oracle.mttkrp(idx, vals, w.dims, facs, n, w.R) for n in range(len(w.dims))]
        np.savez(os.path.join(out_dir, f"t{i}.npz"), *res)
        units += w.nnz * w.R * len(w.dims)
    secs = 0.5 + rank  # rank 1 is the slowest
    thr = multi.aggregate_throughput(secs, units)
    t, u = multi.reduce_timing(secs, units)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([thr, t, u, len(mine)]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    pytest.importorskip("torch.distributed")
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    specs = synth.batched_specs(6, seed0=300, nnz_scale=0.002)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    total_units = sum(w.nnz * w.R * len(w.dims) for w in specs)
    assert r0[3] + r1[3] == len(specs)                      # shards cover the batch
    np.testing.assert_allclose([r0[1], r1[1]], 1.5)         # max of 0.5 and 1.5 s
    np.testing.assert_allclose([r0[2], r1[2]], total_units)  # units summed over ranks
    np.testing.assert_allclose([r0[0], r1[0]], total_units / 1.5)
    for i, w in enumerate(specs):                            # every tensor, same results
        z = np.load(tmp_path / f"t{i}.npz")
        idx, vals = w.coo()
        facs = [f[:, :w.R].astype(np.float64) for f in w.factors()]
        for n in range(len(w.dims)):
            np.testing.assert_array_equal(z[f"arr_{n}"], oracle.mttkrp(idx, vals, w.dims, facs, n, w.R))


def test_shard_is_a_partition():
    import sys
    sys.path.insert(0, ROOT)
    from paper_1809_09175_gb300 import multi
    items = list(range(17))
    parts = [multi.shard(items, r, 4) for r in range(4)]
    assert sorted(sum(parts, [])) == items
    assert all(len(p) in (4, 5) for p in parts)
    assert len({multi.rank_seed(3, r) for r in range(8)}) == 8
    with pytest.raises(ValueError):
        multi.shard(items, 4, 4)

"""Splitting one graph's count over processes: partition by wedge mass, owner
range counts, and the sum across a process group (world_size 2, gloo, CPU).
The per-range counts come from the oracle, so no GPU is needed."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1907_08607_gb300 import shard


def _prefix(wx):
    return np.concatenate([[0], np.cumsum(wx)]).astype(np.uint64)


def test_partition_covers_and_balances():
    rng_prefix = _prefix(np.array([synth.draw(3, 1, i) % 1000 for i in range(5000)], dtype=np.uint64))
    for k in (1, 2, 3, 7, 64):
        parts = shard.partition(rng_prefix, k)
        assert len(parts) == k and parts[0][0] == 0 and parts[-1][1] == 5000
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        masses = [int(rng_prefix[h]) - int(rng_prefix[l]) for l, h in parts]
        assert sum(masses) == int(rng_prefix[-1])
        assert max(masses) - min(masses) <= 2 * 999 + 1       # one owner's mass either side
    # degenerate: more parts than owners, zero mass
    parts = shard.partition(np.zeros(4, np.uint64), 5)
    assert parts[0][0] == 0 and parts[-1][1] == 3


def test_owner_ranges_add_up_to_the_whole():
    g = synth.workload(1)
    full = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    pre = _prefix(oracle.owner_wedges(g.nU, g.nV, g.u, g.v, "degree"))
    assert int(pre[-1]) == full.W
    glob, pv, pe, W = 0, 0, 0, 0
    for lo, hi in shard.partition(pre, 4):
        c = oracle.count_range(g.nU, g.nV, g.u, g.v, lo, hi, "degree")
        assert c.W == int(pre[hi]) - int(pre[lo])
        glob += c.global_count
        W += c.W
        pv = pv + c.per_vertex
        pe = pe + c.per_edge
    assert glob == full.global_count and W == full.W
    np.testing.assert_array_equal(pv, full.per_vertex)
    np.testing.assert_array_equal(pe, full.per_edge)


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.workload(1)
        pre = _prefix(oracle.owner_wedges(g.nU, g.nV, g.u, g.v, "degree"))
        lo, hi = shard.partition(pre, world)[rank]
        c = oracle.count_range(g.nU, g.nV, g.u, g.v, lo, hi, "degree", nthreads=2)
        parts = [torch.tensor([c.global_count], dtype=torch.int64),
                 torch.from_numpy(c.per_vertex.view(np.int64).copy()),
                 torch.from_numpy(c.per_edge.view(np.int64).copy())]
        shard.sum_parts(parts)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.concatenate([p.numpy() for p in parts]).view(np.uint64))
    finally:
        dist.destroy_process_group()


def test_two_process_gloo_sum_equals_single_count(tmp_path):
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    g = synth.workload(1)
    full = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    want = np.concatenate([[full.global_count], full.per_vertex, full.per_edge]).astype(np.uint64)
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"r{r}.npy"), want)

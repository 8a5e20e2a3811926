"""GPU parity at the full workload sizes.

* Chung-Lu |U|=1M, |V|=4M, m=5e7: the launch configuration bench.py times
  (degree ranking, automatic aggregation, default retrieval, all outputs) is
  compared element by element with the complete oracle; every other ranking x
  aggregation x retrieval combination is compared with the same oracle result
  (counts do not depend on the ranking).
* Chung-Lu |U|=20M, |V|=60M, m=3e8, batch aggregation within a 16 GiB scratch
  budget: the oracle's complete outputs (computed once, about half an hour on
  8 cores) are compared through stored SHA-256 digests, plus the counting
  invariants, agreement with a second configuration, and per-vertex /
  per-edge values of sampled vertices and edges evaluated one by one from
  Eq. 1 and Eq. 2.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    pb.load_library()
    return pb


def _sample(seed, hi, k):
    return np.unique(np.array([synth.draw(seed, 11, i) % hi for i in range(k)], dtype=np.uint64))


@pytest.fixture(scope="module")
def cl2():
    g = synth.workload(2)
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    return g, ref


def test_cl2_bench_configuration_matches_oracle(pb, cl2):
    import torch
    g, ref = cl2
    du = torch.from_numpy(g.u.view(np.int32)).cuda()
    dv = torch.from_numpy(g.v.view(np.int32)).cuda()
    G = pb.Graph.from_edges(g.nU, g.nV, du, dv).rank("degree")
    c = G.count_all("auto", on_device=True)
    assert G.wedges == ref.W
    assert c.global_count == ref.global_count
    np.testing.assert_array_equal(c.per_vertex_U.cpu().numpy().view(np.uint64), ref.per_vertex[: g.nU])
    np.testing.assert_array_equal(c.per_vertex_V.cpu().numpy().view(np.uint64), ref.per_vertex[g.nU:])
    np.testing.assert_array_equal(c.per_edge.cpu().numpy().view(np.uint64), ref.per_edge)
    G.free()


@pytest.mark.parametrize("kind", ["side", "degree", "approx_degree"])
def test_cl2_every_aggregation_and_retrieval(pb, cl2, kind):
    g, ref = cl2
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank(kind)
    for rt in ["low", "high"]:
        G.set_retrieval(rt)
        for agg in ["sort", "hash", "hist", "batch", "auto"]:
            c = G.count_all(agg)
            assert c.global_count == ref.global_count, (kind, rt, agg)
            np.testing.assert_array_equal(c.per_vertex_U, ref.per_vertex[: g.nU])
            np.testing.assert_array_equal(c.per_vertex_V, ref.per_vertex[g.nU:])
            np.testing.assert_array_equal(c.per_edge, ref.per_edge)
    G.free()


def test_cl2_sort_reaggregation_matches_oracle(pb, cl2):
    g, ref = cl2
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree").set_butterfly_aggregation("sort")
    for rt in ["low", "high"]:
        G.set_retrieval(rt)
        c = G.count_all("sort")
        assert c.global_count == ref.global_count, rt
        np.testing.assert_array_equal(c.per_vertex_U, ref.per_vertex[: g.nU])
        np.testing.assert_array_equal(c.per_vertex_V, ref.per_vertex[g.nU:])
        np.testing.assert_array_equal(c.per_edge, ref.per_edge)
    G.free()


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


@pytest.fixture(scope="module")
def cl3():
    with open(os.path.join(os.path.dirname(__file__), "golden", "cl3_oracle.json")) as f:
        gold = json.load(f)
    g = synth.workload(3)
    assert (g.nU, g.nV, g.m) == (gold["nU"], gold["nV"], gold["m"])
    return g, gold


def test_cl3_bench_configuration_matches_oracle_digest(pb, cl3):
    """The launch configuration bench.py times by default: device-resident
    edge list, degree ranking, global + per-edge counts, batch aggregation
    within 16 GiB; the per-edge array must hash to the oracle's digest."""
    import torch
    g, gold = cl3
    du = torch.from_numpy(g.u.view(np.int32)).cuda()
    dv = torch.from_numpy(g.v.view(np.int32)).cuda()
    for _ in range(2):  # a second count on a fresh graph reuses the memory pool
        G = pb.Graph.from_edges(g.nU, g.nV, du, dv).rank("degree")
        assert G.wedges == gold["W"]
        c = G.count_all("batch", scratch_bytes=16 << 30, vertex=False, edge=True, on_device=True)
        G.free()
        assert c.global_count == gold["global"]
        assert _digest(c.per_edge.cpu().numpy().view(np.uint64)) == gold["per_edge_sha256"]
    del du, dv, c
    torch.cuda.empty_cache()


def test_cl3_batch_16gib_matches_oracle_digests_invariants_and_samples(pb, cl3):
    """Complete oracle outputs on this workload are stored as SHA-256 digests
    (tests/golden/cl3_oracle.json, written by tests/golden/make_cl3_oracle.py
    from oracle.count); the GPU's per-vertex and per-edge arrays must hash to
    the same values, and W and the global count must be equal."""
    g, gold = cl3
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    assert G.info().m == g.m
    assert G.wedges == gold["W"]
    c = G.count_all("batch", scratch_bytes=16 << 30)
    assert c.global_count == gold["global"]
    assert _digest(np.concatenate([c.per_vertex_U, c.per_vertex_V])) == gold["per_vertex_sha256"]
    assert _digest(c.per_edge) == gold["per_edge_sha256"]
    G.set_retrieval("low")
    c2 = G.count_all("auto", glob=True, vertex=True, edge=False)
    G.free()
    gl = c.global_count
    assert gl > 0 and gl == c2.global_count
    np.testing.assert_array_equal(c.per_vertex_U, c2.per_vertex_U)
    np.testing.assert_array_equal(c.per_vertex_V, c2.per_vertex_V)
    assert int(c.per_vertex_U.sum(dtype=np.uint64)) == 2 * gl
    assert int(c.per_vertex_V.sum(dtype=np.uint64)) == 2 * gl
    assert int(c.per_edge.sum(dtype=np.uint64)) == 4 * gl
    qv = _sample(0xC3, g.nU + g.nV, 200)
    want_v = oracle.vertex_eq1(g.nU, g.nV, g.u, g.v, qv)
    pv = np.concatenate([c.per_vertex_U, c.per_vertex_V])
    np.testing.assert_array_equal(pv[qv.astype(np.int64)], want_v)
    qe = _sample(0xE3, g.m, 200)
    want_e = oracle.edge_eq2(g.nU, g.nV, g.u, g.v, qe)
    np.testing.assert_array_equal(c.per_edge[qe.astype(np.int64)], want_e)

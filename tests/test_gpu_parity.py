"""GPU path vs the CPU oracle, element by element (uint64, bit-exact).

Every call goes through the C ABI (libpb.so) via the Python binding.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._fixtures import fig2_graph, fig2_rank, random_rank, tiny_graphs

pytestmark = pytest.mark.gpu

RANKS = ["side", "degree", "approx_degree", "complement_degeneracy", "approx_complement_degeneracy"]
AGGS = ["hash", "hist", "batch", "sort", "auto"]


@pytest.fixture(scope="module")
def pb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    pb.load_library()
    return pb


RETRIEVALS = ["low", "high"]


def _gpu_all(pb, g, kind, agg, rank_of=None, scratch=0, retrieval="auto"):
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v)
    if rank_of is not None:
        G.rank_custom(rank_of)
    else:
        G.rank(kind)
    G.set_retrieval(retrieval)
    c = G.count_all(agg, scratch_bytes=scratch)
    W = G.wedges
    ranks = G.ranks()
    G.free()
    return c, W, ranks


def _assert_same(c, ref, nU):
    assert c.global_count == ref.global_count
    np.testing.assert_array_equal(c.per_vertex_U, ref.per_vertex[:nU])
    np.testing.assert_array_equal(c.per_vertex_V, ref.per_vertex[nU:])
    np.testing.assert_array_equal(c.per_edge, ref.per_edge)


def test_fig2_worked_example(pb, fig2):
    nU, nV, u, v, gid = fig2_graph(fig2)
    rk = fig2_rank(fig2, gid)
    ref = oracle.count(nU, nV, u, v, rank_of=rk)
    for agg, rt in [(a, r) for a in AGGS for r in RETRIEVALS]:
        c, W, ranks = _gpu_all(pb, synth.Graph(nU, nV, u, v), None, agg, rank_of=rk, retrieval=rt)
        assert W == 6
        np.testing.assert_array_equal(ranks, rk)
        _assert_same(c, ref, nU)
        assert c.global_count == 3


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (7, 4), (33, 5), (40, 40)])
def test_complete_bipartite(pb, a, b):
    g = synth.complete_bipartite(a, b)
    C2 = lambda x: x * (x - 1) // 2  # noqa: E731
    for kind in RANKS:
        for agg, rt in [(x, r) for x in AGGS for r in RETRIEVALS]:
            c, _, _ = _gpu_all(pb, g, kind, agg, retrieval=rt)
            assert c.global_count == C2(a) * C2(b)
            assert np.all(c.per_vertex_U == (a - 1) * C2(b))
            assert np.all(c.per_vertex_V == (b - 1) * C2(a))
            assert np.all(c.per_edge == (a - 1) * (b - 1))


def test_tiny_graphs_every_ranking_and_aggregation(pb):
    for i, g in enumerate(tiny_graphs(24)):
        ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
        for kind in RANKS + ["random"]:
            rk = random_rank(500 + i, g.nU + g.nV) if kind == "random" else None
            for agg, rt in [(x, r) for x in AGGS for r in RETRIEVALS]:
                c, W, ranks = _gpu_all(pb, g, kind, agg, rank_of=rk, retrieval=rt)
                _assert_same(c, ref, g.nU)
                want_W = oracle.wedges(g.nU, g.nV, g.u, g.v, kind=kind if rk is None else "side", rank_of=rk)
                assert W == want_W
                if rk is None:
                    np.testing.assert_array_equal(ranks, oracle.rank(g.nU, g.nV, g.u, g.v, kind))


@pytest.fixture(scope="module")
def er1():
    return synth.workload(1)


def test_er_workload_degree_hash(pb, er1):
    """The ER 2k x 3k workload: exact degree ranking, hash aggregation,
    global + per-vertex counts."""
    g = er1
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    assert G.wedges == ref.W
    np.testing.assert_array_equal(G.ranks(), oracle.rank(g.nU, g.nV, g.u, g.v, "degree"))
    assert G.count_global("hash") == ref.global_count
    U, V = G.count_vertex("hash")
    np.testing.assert_array_equal(U, ref.per_vertex[: g.nU])
    np.testing.assert_array_equal(V, ref.per_vertex[g.nU:])
    G.free()


def test_er_workload_all_combinations(pb, er1):
    g = er1
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    for kind in RANKS:
        W = oracle.wedges(g.nU, g.nV, g.u, g.v, kind=kind)
        for agg in AGGS:
            c, gW, _ = _gpu_all(pb, g, kind, agg)
            assert gW == W
            _assert_same(c, ref, g.nU)


@pytest.fixture(scope="module")
def mid():
    """Skewed Chung-Lu graphs large enough that every work tier is populated
    (first endpoints with a few, a few thousand and hundreds of thousands of
    wedges), plus a ragged ER graph."""
    return [
        synth.chung_lu_graph(0xC0FFEE, 20_000, 60_000, 400_000, 2.1, 2.5, cap_u=3000, cap_v=3000),
        synth.chung_lu_graph(0xBEEF, 30_000, 10_000, 300_000, 2.0, 2.0, cap_u=2500, cap_v=2500),
        synth.er_graph(0xABC, 3_001, 977, 60_013),
    ]


def test_mid_graphs_all_combinations(pb, mid):
    for g in mid:
        ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
        for kind in RANKS:
            W = oracle.wedges(g.nU, g.nV, g.u, g.v, kind=kind)
            for agg, rt in [(x, r) for x in AGGS for r in RETRIEVALS]:
                c, gW, _ = _gpu_all(pb, g, kind, agg, retrieval=rt)
                assert gW == W, (g.name, kind, agg, rt)
                _assert_same(c, ref, g.nU)


def test_small_scratch_budget_chunks_exactly(pb, mid):
    """A budget that holds a single unit of work (one device-memory slot, or
    one first endpoint's wedges for sort) forces many rounds; counts stay
    exact.  A budget below one unit is refused with PB_ERR_SCRATCH."""
    g = mid[0]
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    n = g.nU + g.nV
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    maxw = G.info().max_wedges_x1
    assert maxw * 40 < G.wedges * 40 // 4          # sort needs several chunks
    for rt in RETRIEVALS:
        G.set_retrieval(rt)
        for agg, budget in [("hist", 8 * n + 4096), ("batch", 8 * n + 4096), ("hash", 32 * n + 4096),
                            ("sort", 40 * maxw + 4096), ("auto", 8 * n + 4096)]:
            c = G.count_all(agg, scratch_bytes=budget)
            _assert_same(c, ref, g.nU)
    G.set_retrieval("low")
    with pytest.raises(pb.PBError) as ei:
        G.count_all("sort", scratch_bytes=maxw)
    assert ei.value.status == 4
    with pytest.raises(pb.PBError) as ei:
        G.count_all("hist", scratch_bytes=1024)
    assert ei.value.status == 4
    G.free()


def test_duplicates_and_device_inputs(pb, er1):
    import torch
    d = synth.with_duplicates(er1, seed=5, frac=0.3)
    ref = oracle.count(d.nU, d.nV, d.u, d.v, kind="approx_degree")
    G = pb.Graph.from_edges(d.nU, d.nV, torch.from_numpy(d.u.view(np.int32)).cuda(),
                            torch.from_numpy(d.v.view(np.int32)).cuda())
    assert G.info().m == er1.m and G.info().m_in == d.m
    G.rank("approx_degree")
    c = G.count_all("auto", on_device=True)
    assert c.global_count == ref.global_count
    np.testing.assert_array_equal(c.per_edge.cpu().numpy().view(np.uint64), ref.per_edge)
    np.testing.assert_array_equal(c.per_vertex_U.cpu().numpy().view(np.uint64), ref.per_vertex[: d.nU])
    np.testing.assert_array_equal(c.per_vertex_V.cpu().numpy().view(np.uint64), ref.per_vertex[d.nU:])
    G.free()


def test_side_ranking_until_ranked(pb, er1):
    """Before pb_rank the graph behaves as side-ranked (computed on first use):
    every query and count sees the side order's wedges and exact counts; a
    pb_rank straight after construction replaces it."""
    g = er1
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    W_side = oracle.wedges(g.nU, g.nV, g.u, g.v, kind="side")
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v)
    inf = G.info()
    assert inf.rank_kind == 0 and inf.W == W_side
    np.testing.assert_array_equal(G.ranks(), oracle.rank(g.nU, g.nV, g.u, g.v, "side"))
    _assert_same(G.count_all("hash"), ref, g.nU)
    G.free()
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v)
    _assert_same(G.count_all("hist"), ref, g.nU)     # a count first
    assert G.wedges == W_side
    G.free()
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    assert G.wedges == oracle.wedges(g.nU, g.nV, g.u, g.v, kind="degree")
    _assert_same(G.count_all("auto"), ref, g.nU)
    G.free()


def test_degenerate_inputs(pb):
    e = np.zeros(0, np.uint32)
    G = pb.Graph.from_edges(3, 4, e, e)
    assert G.wedges == 0 and G.count_global() == 0
    U, V = G.count_vertex()
    assert np.all(U == 0) and np.all(V == 0)
    assert G.count_edge().shape == (0,)
    G.free()
    # a star: wedges, no butterflies
    G = pb.Graph.from_edges(1, 50, np.zeros(50, np.uint32), np.arange(50, dtype=np.uint32))
    for kind in RANKS:
        G.rank(kind)
        assert G.count_global("hist") == 0
        assert np.all(G.count_edge("hash") == 0)
    G.free()
    # one edge
    G = pb.Graph.from_edges(1, 1, np.zeros(1, np.uint32), np.zeros(1, np.uint32)).rank("degree")
    assert G.count_global() == 0 and G.wedges == 0
    G.free()
    # one empty side, and isolated vertices only: no wedges, all counts zero
    for nU, nV in [(0, 5), (5, 0), (1, 1)]:
        G = pb.Graph.from_edges(nU, nV, e, e)
        for kind in RANKS:
            G.rank(kind)
            assert G.wedges == 0 and G.count_global() == 0
            U, V = G.count_vertex()
            assert U.shape == (nU,) and V.shape == (nV,) and not U.any() and not V.any()
        G.free()
    with pytest.raises(pb.PBError) as ei:  # no vertices at all
        pb.Graph.from_edges(0, 0, e, e)
    assert ei.value.status == 1
    # invalid ids / rankings are rejected with PB_ERR_INVALID
    with pytest.raises(pb.PBError) as ei:
        pb.Graph.from_edges(2, 2, np.array([0, 2], np.uint32), np.array([0, 1], np.uint32))
    assert ei.value.status == 1
    G = pb.Graph.from_edges(2, 2, np.array([0, 1], np.uint32), np.array([0, 1], np.uint32))
    with pytest.raises(pb.PBError):
        G.rank_custom(np.array([0, 0, 1, 2], np.uint32))
    G.free()


def test_virtual_shards_sum_to_the_whole(pb, mid):
    """k owner ranges of equal wedge mass on one GPU: the partial counts add
    up, element by element, to the unsharded count."""
    from paper_1907_08607_gb300 import shard
    g = mid[1]
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    for rt in RETRIEVALS:
        G.set_retrieval(rt)
        pre = G.wedge_prefix()
        assert int(pre[-1]) == G.wedges
        for agg in ["auto", "sort"]:
            for k in (1, 3, 8):
                tot_g, pv, pe = 0, 0, 0
                for lo, hi in shard.partition(pre, k):
                    c = G.count_all(agg, owners=(lo, hi))
                    tot_g += c.global_count
                    pv = pv + np.concatenate([c.per_vertex_U, c.per_vertex_V])
                    pe = pe + c.per_edge
                assert tot_g == ref.global_count
                np.testing.assert_array_equal(pv, ref.per_vertex)
                np.testing.assert_array_equal(pe, ref.per_edge)
    G.free()


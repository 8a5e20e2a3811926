"""Butterfly aggregation by re-aggregation (Sec. "Butterfly aggregation"):
per-vertex and per-edge contributions sorted by key and summed per key
instead of atomic adds.  Counts must equal the oracle's bit for bit, under
every ranking and retrieval, for each subset of outputs, and across chunks
when the scratch budget splits the wedges.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._fixtures import fig2_graph, fig2_rank, tiny_graphs

pytestmark = pytest.mark.gpu

RANKS = ["side", "degree", "approx_degree", "complement_degeneracy", "approx_complement_degeneracy"]
# Scratch bytes per wedge the sort path asks for with re-aggregation of both
# outputs; a budget of this times the largest owner's wedges is the smallest
# one accepted.
RE_BYTES_PER_WEDGE = 40 + 2 * (32 + 52)


@pytest.fixture(scope="module")
def pb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    pb.load_library()
    return pb


def _count(pb, g, kind, retrieval="auto", rank_of=None, scratch=0, vertex=True, edge=True):
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v)
    G.rank_custom(rank_of) if rank_of is not None else G.rank(kind)
    G.set_retrieval(retrieval).set_butterfly_aggregation("sort")
    c = G.count_all("sort", scratch_bytes=scratch, vertex=vertex, edge=edge)
    G.free()
    return c


def _same(c, ref, nU, vertex=True, edge=True):
    assert c.global_count == ref.global_count
    if vertex:
        np.testing.assert_array_equal(c.per_vertex_U, ref.per_vertex[:nU])
        np.testing.assert_array_equal(c.per_vertex_V, ref.per_vertex[nU:])
    if edge:
        np.testing.assert_array_equal(c.per_edge, ref.per_edge)


def test_fig2_worked_example(pb, fig2):
    nU, nV, u, v, gid = fig2_graph(fig2)
    rk = fig2_rank(fig2, gid)
    ref = oracle.count(nU, nV, u, v, rank_of=rk)
    for rt in ["low", "high"]:
        _same(_count(pb, synth.Graph(nU, nV, u, v), None, rt, rank_of=rk), ref, nU)


def test_tiny_graphs_every_ranking_and_output_subset(pb):
    for i, g in enumerate(tiny_graphs(24)):
        ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
        for kind in RANKS:
            for rt in ["low", "high"]:
                for vertex, edge in [(True, True), (True, False), (False, True)]:
                    c = _count(pb, g, kind, rt, vertex=vertex, edge=edge)
                    _same(c, ref, g.nU, vertex, edge)


@pytest.fixture(scope="module")
def skewed():
    return [
        synth.chung_lu_graph(0xC0FFEE, 20_000, 60_000, 400_000, 2.1, 2.5, cap_u=3000, cap_v=3000),
        synth.er_graph(0xABC, 3_001, 977, 60_013),
    ]


def test_skewed_graphs_match_atomic_path_and_oracle(pb, skewed):
    for g in skewed:
        ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
        for kind in ["degree", "side"]:
            for rt in ["low", "high"]:
                _same(_count(pb, g, kind, rt), ref, g.nU)


def test_many_chunks_stay_exact(pb, skewed):
    """A budget that holds one owner's wedges forces one chunk per few owners;
    every chunk re-aggregates its own pairs into the same counters."""
    g = skewed[0]
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree").set_butterfly_aggregation("sort")
    for rt in ["low", "high"]:
        G.set_retrieval(rt)
        maxw = int(np.diff(G.wedge_prefix()).max())
        budget = RE_BYTES_PER_WEDGE * max(maxw, G.wedges // 9) + 4096
        _same(G.count_all("sort", scratch_bytes=budget), ref, g.nU)
    G.free()


def test_needs_sort_wedge_aggregation(pb, skewed):
    g = skewed[1]
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree").set_butterfly_aggregation("sort")
    for agg in ["hash", "hist", "batch", "auto"]:
        with pytest.raises(pb.PBError) as ei:
            G.count_all(agg)
        assert ei.value.status == 1
    G.set_butterfly_aggregation("atomic")
    assert G.count_all("hash", vertex=False, edge=False).global_count == G.count_all("sort").global_count
    with pytest.raises(pb.PBError) as ei:
        pb._check(pb.load_library().pb_set_butterfly_aggregation(G._h, 7))
    assert ei.value.status == 1
    G.free()

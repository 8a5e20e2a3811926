"""The autotuner (pb_autotune / pb_set_plan): its statistics agree with the
wedge prefix the library exposes, its choice follows the scratch budget, and
counts under every plan -- chosen or pinned, in one graph or across a batch
whose graphs took different plans -- equal the oracle's."""
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


@pytest.fixture(scope="module")
def skewed():
    g = synth.chung_lu_graph(0xA770, 30_000, 90_000, 600_000, 2.0, 2.0, cap_u=5000, cap_v=5000)
    return g, oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")


def _check(c, ref, g):
    assert c.global_count == ref.global_count
    np.testing.assert_array_equal(c.per_vertex_U, ref.per_vertex[: g.nU])
    np.testing.assert_array_equal(c.per_vertex_V, ref.per_vertex[g.nU:])
    np.testing.assert_array_equal(c.per_edge, ref.per_edge)


def test_plan_statistics_match_the_wedge_prefix(pb, skewed):
    g, ref = skewed
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    p = G.autotune()
    G.set_retrieval(p["retrieval"])
    wc = np.diff(G.wedge_prefix().astype(np.int64))
    tiers = [(wc >= 1) & (wc <= p["light_max"]), (wc > p["light_max"]) & (wc <= p["med_max"]),
             (wc > p["med_max"]) & (wc <= p["large_max"]), wc > p["large_max"]]
    assert p["owners"] == [int(t.sum()) for t in tiers]
    assert p["wedges"] == [int(wc[t].sum()) for t in tiers]
    assert sum(p["wedges"]) == G.wedges == ref.W and p["max_owner_wedges"] == int(wc.max())
    # a wedge's second endpoint owns it in the other direction: the hot share
    # is the other direction's wedges held by the first `hot` labels of each side
    G.set_retrieval("low" if p["retrieval"] == "high" else "high")
    wo = np.diff(G.wedge_prefix().astype(np.int64))
    H = p["hot"]
    hot = wo[: min(H, g.nU)].sum() + wo[g.nU: g.nU + min(H, g.nV)].sum()
    assert p["hot_hit"] == pytest.approx(hot / G.wedges, rel=1e-12)
    assert p["agg"] in ("batch", "hash", "hist") and p["light_max"] <= 768 and p["med_max"] <= 4096
    assert p["med_max"] <= p["large_max"] <= 65535
    # mid-size owners' mean wedges per neighbour (the owner's degree under
    # high retrieval), and the tier it selects for them
    G.set_retrieval(p["retrieval"])
    deg = np.diff(G.layout()["off"].cpu().numpy().view(np.uint32).astype(np.int64))
    span = deg if p["retrieval"] == "high" else None
    if span is not None:
        mid = (wc > p["light_max"]) & (wc <= 65535)
        assert p["mid_segment"] == pytest.approx(wc[mid].sum() / max(span[mid].sum(), 1), rel=1e-12)
    assert p["med_max"] == (p["light_max"] if p["mid_segment"] >= 80 else 4096) and p["large_max"] == 4096
    G.free()


def _rule(p, budget):
    """The documented choice for a plan's statistics and a budget."""
    if p["owners"][3] == 0:
        return "batch"
    want = min(p["resident_blocks"], p["owners"][3])
    fit_d = budget // (p["slot_bytes_dense"] + 16)
    fit_h = budget // (p["slot_bytes_hash"] + 16)
    if p["agg"] == "hist":
        return "hist"
    return "batch" if fit_d >= want or fit_d >= fit_h else "hash"


@pytest.fixture(scope="module")
def with_heavy():
    """A graph whose largest owners pass the large tier's bound (16384 wedges)."""
    g = synth.chung_lu_graph(0xA771, 100_000, 300_000, 3_000_000, 2.0, 2.0, cap_u=20000, cap_v=20000)
    return g, oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")


def test_choice_follows_the_budget_and_counts_stay_exact(pb, with_heavy):
    """The aggregation follows the documented rule at budgets on either side
    of the dense slots' need; every choice, and every explicit aggregation
    under a tiny budget, counts exactly."""
    g, ref = with_heavy
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    big = G.autotune(16 << 30)
    assert big["owners"][3] > 0 and big["agg"] == _rule(big, 16 << 30) == "batch"
    want = min(big["resident_blocks"], big["owners"][3])
    for budget in (16 << 30, want * (big["slot_bytes_dense"] + 16), want * (big["slot_bytes_dense"] + 16) - 1,
                   8 * (big["slot_bytes_dense"] + 16)):
        p = G.autotune(budget)
        assert p["agg"] == _rule(p, budget), budget
        assert p["slot_bytes"] == (p["slot_bytes_hash"] if p["agg"] == "hash" else p["slot_bytes_dense"])
        _check(G.count_all("auto", scratch_bytes=budget), ref, g)
    tiny = 4 * (max(big["slot_bytes_hash"], big["slot_bytes_dense"]) + 16)   # four slots: clusters share them
    for agg in ("hist", "batch", "hash"):
        _check(G.count_all(agg, scratch_bytes=tiny), ref, g)
    G.free()


@pytest.mark.parametrize("edit", [dict(agg="hash"), dict(agg="hist", hub_cluster=4, hub_min=0),
                                  dict(agg="batch", hot=0), dict(agg="batch", hot=49152),
                                  dict(agg="hash", hot=1000), dict(light_max=1, med_max=1, large_max=1),
                                  dict(light_max=100, med_max=300, large_max=2000),
                                  dict(med_max=768, large_max=65535), dict(large_max=4096),
                                  dict(retrieval="low"), dict(retrieval="low", large_max=65535)])
def test_every_pinned_plan_counts_exactly(pb, skewed, edit):
    g, ref = skewed
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    p = G.autotune()
    p.update(edit)
    G.set_plan(p)
    _check(G.count_all("auto"), ref, g)
    assert G.count_all("auto", vertex=False, edge=False).global_count == ref.global_count
    c = G.count_all("auto", vertex=True, edge=False)
    assert c.global_count == ref.global_count
    np.testing.assert_array_equal(c.per_vertex_U, ref.per_vertex[: g.nU])
    c = G.count_all("auto", vertex=False, edge=True)
    np.testing.assert_array_equal(c.per_edge, ref.per_edge)
    G.set_plan(None)
    G.free()


def test_pinned_plan_is_validated(pb, skewed):
    g, _ = skewed
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    p = G.autotune()
    for bad in (dict(agg="sort"), dict(agg="auto"), dict(retrieval="auto"), dict(hub_cluster=0),
                dict(hub_cluster=17)):
        q = dict(p, **bad)
        with pytest.raises(pb.PBError) as ei:
            G.set_plan(q)
        assert ei.value.status == 1
    G.free()


def test_batch_graphs_on_different_plans(pb):
    """Graphs of one batch on different heavy paths -- half pinned to the
    hashed cold part, half to the dense histogram, some with moved tier
    bounds -- each equal their count alone and the oracle's."""
    gs = [synth.batch_graph(i, m_hi=3e5) for i in range(40)]
    big = synth.chung_lu_graph(0xA770, 30_000, 90_000, 600_000, 2.0, 2.0, cap_u=5000, cap_v=5000)
    gs.insert(7, big)
    Gs = [pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree") for g in gs]
    for i, G in enumerate(Gs):
        p = G.autotune()
        p["agg"] = "hash" if i % 2 else "batch"
        if i % 3 == 0:
            p["large_max"] = 4096 if i % 2 else 65535
        G.set_plan(p)
    alone = [G.count_all("auto", edge=False) for G in Gs]
    B = pb.Batch(Gs, vertex=True)
    for _ in range(2):
        B.run()
        glob = B.globals()
        for i in range(len(gs)):
            assert int(glob[i]) == alone[i].global_count, i
            U, V = B.vertex_counts(i)
            np.testing.assert_array_equal(U, alone[i].per_vertex_U)
            np.testing.assert_array_equal(V, alone[i].per_vertex_V)
    for i in list(range(0, len(gs), 5)) + [7]:
        ref = oracle.count(gs[i].nU, gs[i].nV, gs[i].u, gs[i].v, per_edge=False)
        assert int(glob[i]) == ref.global_count
        np.testing.assert_array_equal(np.concatenate(B.vertex_counts(i)), ref.per_vertex)
    B.free()
    B = pb.Batch(Gs, vertex=False)                 # global counts only
    B.run()
    assert [int(x) for x in B.globals()] == [c.global_count for c in alone]
    B.free()
    for G in Gs:
        G.free()

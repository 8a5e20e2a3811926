"""Pins of the CPU oracle to things other than itself (no GPU needed).

* the paper's worked example (Figs. 1-2, golden fixture);
* closed forms on complete bipartite graphs K_{a,b};
* brute force over all vertex pairs (the definitions) on seeded tiny graphs;
* counting invariants (each butterfly has two vertices per side and four
  edges) and invariance of the counts under every ranking;
* the retrieved-wedge count: brute-force wedge listing, and the closed form
  under side order;
* per-edge values straight from Eq. 2, edge by edge.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import brute
from tests._fixtures import fig2_graph, fig2_rank, random_rank, tiny_graphs

RANKS = ["side", "degree", "approx_degree"]


# ----------------------------------------------------------------- Figs. 1-2
def test_fig2_worked_example(fig2):
    nU, nV, u, v, gid = fig2_graph(fig2)
    rk = fig2_rank(fig2, gid)
    c = oracle.count(nU, nV, u, v, rank_of=rk)
    assert c.W == len(fig2["wedges_step2"]) == 6
    assert c.global_count == fig2["global"] == 3
    for name, val in fig2["per_vertex_step4"].items():
        assert int(c.per_vertex[gid[name]]) == val, name
    for k, (a, b) in enumerate(fig2["edges"]):
        assert int(c.per_edge[k]) == fig2["per_edge_from_fig1"][f"{a}-{b}"]
    # the same numbers from the definitions
    g, pv, pe = brute.counts(nU, nV, u, v)
    assert g == 3
    assert [int(x) for x in pv] == [int(x) for x in c.per_vertex]
    assert [int(x) for x in pe] == [int(x) for x in c.per_edge]
    assert brute.wedges(nU, nV, u, v, rk) == 6
    assert oracle.wedges(nU, nV, u, v, rank_of=rk) == 6
    listed = brute.butterflies_listed(nU, nV, u, v)
    U, V = fig2["vertices"]["U"], fig2["vertices"]["V"]
    want = sorted(((U.index(a1), U.index(a2)), tuple(sorted((V.index(b1), V.index(b2)))))
                  for (a1, a2), (b1, b2) in fig2["butterflies"])
    assert sorted(listed) == want


def test_fig2_counts_same_under_every_ranking(fig2):
    nU, nV, u, v, gid = fig2_graph(fig2)
    for kind in RANKS:
        c = oracle.count(nU, nV, u, v, kind=kind)
        assert c.global_count == 3
        assert {n: int(c.per_vertex[gid[n]]) for n in gid} == fig2["per_vertex_step4"]


# ----------------------------------------------------------------- K_{a,b}
@pytest.mark.parametrize("a,b", [(1, 1), (1, 5), (5, 1), (2, 2), (2, 3), (3, 2), (4, 7), (9, 6),
                                 (12, 12), (30, 3)])
@pytest.mark.parametrize("kind", RANKS)
def test_complete_bipartite_closed_forms(a, b, kind):
    g = synth.complete_bipartite(a, b)
    c = oracle.count(a, b, g.u, g.v, kind=kind)
    C2 = lambda x: x * (x - 1) // 2  # noqa: E731
    assert c.global_count == C2(a) * C2(b)
    assert np.all(c.per_vertex[:a] == (a - 1) * C2(b))
    assert np.all(c.per_vertex[a:] == (b - 1) * C2(a))
    assert np.all(c.per_edge == (a - 1) * (b - 1))


def test_complete_bipartite_brute():
    for a, b in [(2, 3), (4, 4), (5, 2)]:
        g = synth.complete_bipartite(a, b)
        glob, pv, pe = brute.counts(a, b, g.u, g.v)
        assert glob == math.comb(a, 2) * math.comb(b, 2)
        assert np.all(pv[:a] == (a - 1) * math.comb(b, 2))
        assert np.all(pv[a:] == (b - 1) * math.comb(a, 2))
        assert np.all(pe == (a - 1) * (b - 1))


# ----------------------------------------------------------------- brute force
@pytest.fixture(scope="module")
def tiny():
    return tiny_graphs(60)


def test_oracle_matches_brute_force_on_tiny_graphs(tiny):
    for i, g in enumerate(tiny):
        glob, pv, pe = brute.counts(g.nU, g.nV, g.u, g.v)
        kinds = RANKS + [random_rank(1000 + i, g.nU + g.nV)]
        for kind in kinds:
            if isinstance(kind, str):
                c = oracle.count(g.nU, g.nV, g.u, g.v, kind=kind, nthreads=1 + i % 3)
                rk = oracle.rank(g.nU, g.nV, g.u, g.v, kind)
            else:
                rk = kind
                c = oracle.count(g.nU, g.nV, g.u, g.v, rank_of=rk, nthreads=2)
            assert c.global_count == glob, (g.name, kind)
            np.testing.assert_array_equal(c.per_vertex.astype(np.int64), pv)
            np.testing.assert_array_equal(c.per_edge.astype(np.int64), pe)
            bw = brute.wedges(g.nU, g.nV, g.u, g.v, rk)
            assert c.W == bw, (g.name, kind)
            assert oracle.wedges(g.nU, g.nV, g.u, g.v, rank_of=rk) == bw


def test_oracle_matches_brute_force_on_1000_more_tiny_graphs():
    """A thousand further seeded tiny graphs (ER and Chung-Lu, up to 31 x 31),
    every ranking: global, per-vertex and per-edge counts equal the
    definitions, and W equals the brute-force wedge count."""
    for i, g in enumerate(tiny_graphs(1000, seed=0x51A8)):
        glob, pv, pe = brute.counts(g.nU, g.nV, g.u, g.v)
        for kind in RANKS:
            c = oracle.count(g.nU, g.nV, g.u, g.v, kind=kind, nthreads=1)
            assert c.global_count == glob, (g.name, kind)
            np.testing.assert_array_equal(c.per_vertex.astype(np.int64), pv)
            np.testing.assert_array_equal(c.per_edge.astype(np.int64), pe)
            assert c.W == brute.wedges(g.nU, g.nV, g.u, g.v, oracle.rank(g.nU, g.nV, g.u, g.v, kind)), (g.name, kind)


def test_eq1_direct_matches_brute(tiny):
    for g in tiny[:20]:
        _, pv, _ = brute.counts(g.nU, g.nV, g.u, g.v)
        q = np.arange(g.nU + g.nV, dtype=np.uint64)
        np.testing.assert_array_equal(oracle.vertex_eq1(g.nU, g.nV, g.u, g.v, q).astype(np.int64), pv)


def test_eq2_direct_matches_brute(tiny):
    for g in tiny[:20]:
        _, _, pe = brute.counts(g.nU, g.nV, g.u, g.v)
        q = np.arange(g.m, dtype=np.uint64)
        np.testing.assert_array_equal(oracle.edge_eq2(g.nU, g.nV, g.u, g.v, q).astype(np.int64), pe)


# ----------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def er1():
    return synth.workload(1)


def test_er_workload_invariants_and_brute(er1):
    g = er1
    cs = {k: oracle.count(g.nU, g.nV, g.u, g.v, kind=k) for k in RANKS}
    ref = cs["degree"]
    for k, c in cs.items():
        assert c.global_count == ref.global_count
        np.testing.assert_array_equal(c.per_vertex, ref.per_vertex)
        np.testing.assert_array_equal(c.per_edge, ref.per_edge)
    G = ref.global_count
    assert G > 0
    assert int(ref.per_vertex[: g.nU].sum()) == 2 * G
    assert int(ref.per_vertex[g.nU:].sum()) == 2 * G
    assert int(ref.per_edge.sum()) == 4 * G          # input has no duplicates
    glob, pv, pe = brute.counts(g.nU, g.nV, g.u, g.v)
    assert glob == G
    np.testing.assert_array_equal(ref.per_vertex.astype(np.int64), pv)
    np.testing.assert_array_equal(ref.per_edge.astype(np.int64), pe)


def test_side_order_wedge_closed_form(er1, tiny):
    """Under side order with endpoints on side X, every pair of neighbours of
    every centre on the other side is retrieved: W = sum C(deg y, 2)."""
    for g in [er1] + tiny[:30]:
        du = np.bincount(g.u, minlength=g.nU).astype(object)
        dv = np.bincount(g.v, minlength=g.nV).astype(object)
        w_endpoints_u = sum(d * (d - 1) // 2 for d in dv)
        w_endpoints_v = sum(d * (d - 1) // 2 for d in du)
        W = oracle.wedges(g.nU, g.nV, g.u, g.v, kind="side")
        assert W == min(w_endpoints_u, w_endpoints_v)
        assert oracle.count(g.nU, g.nV, g.u, g.v, kind="side", per_edge=False).W == W


def test_side_order_wedges_do_not_depend_on_the_order_inside_a_side(tiny):
    """The order inside each side (a reading: the paper fixes only which side
    comes first) changes neither W nor the counts: any side-first ranking with
    a random order inside the sides retrieves the same wedges, checked against
    brute force."""
    for i, g in enumerate(tiny[:30]):
        n = g.nU + g.nV
        side = oracle.rank(g.nU, g.nV, g.u, g.v, "side")
        u_first = g.nU > 0 and int(side[: g.nU].min()) == 0   # U holds rank 0
        perm = random_rank(900 + i, n).astype(np.int64)
        first = np.arange(g.nU) if u_first else np.arange(g.nU, n)
        second = np.arange(g.nU, n) if u_first else np.arange(g.nU)
        order = np.concatenate([first[np.argsort(perm[first], kind="stable")],
                                second[np.argsort(perm[second], kind="stable")]])
        rk = np.empty(n, np.uint32)
        rk[order] = np.arange(n, dtype=np.uint32)
        W = oracle.wedges(g.nU, g.nV, g.u, g.v, kind="side")
        assert oracle.wedges(g.nU, g.nV, g.u, g.v, rank_of=rk) == W
        assert brute.wedges(g.nU, g.nV, g.u, g.v, rk) == W
        ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="side")
        c = oracle.count(g.nU, g.nV, g.u, g.v, rank_of=rk)
        assert c.global_count == ref.global_count
        np.testing.assert_array_equal(c.per_vertex, ref.per_vertex)
        np.testing.assert_array_equal(c.per_edge, ref.per_edge)


def test_rank_orders_have_their_defining_property(er1, tiny):
    for g in [er1] + tiny[:20]:
        n = g.nU + g.nV
        deg = np.concatenate([np.bincount(g.u, minlength=g.nU), np.bincount(g.v, minlength=g.nV)])
        for kind in RANKS:
            r = oracle.rank(g.nU, g.nV, g.u, g.v, kind).astype(np.int64)
            assert np.array_equal(np.sort(r), np.arange(n))       # a permutation
            order = np.empty(n, np.int64)
            order[r] = np.arange(n)
            if kind == "degree":
                d = deg[order]
                assert np.all(d[:-1] >= d[1:])                    # decreasing degree
                tie = d[:-1] == d[1:]
                assert np.all(order[:-1][tie] < order[1:][tie])   # ties by id
            elif kind == "approx_degree":
                lg = np.where(deg > 0, np.floor(np.log2(np.maximum(deg, 1))), -1)[order]
                assert np.all(lg[:-1] >= lg[1:])                  # decreasing log-degree
                tie = lg[:-1] == lg[1:]
                assert np.all(order[:-1][tie] < order[1:][tie])   # original order kept
            else:
                side = (order >= g.nU).astype(np.int64)
                assert np.all(np.diff(side) >= 0) or np.all(np.diff(side) <= 0)  # one side first
                wu = sum(int(x) * (int(x) - 1) // 2 for x in deg[g.nU:])
                wv = sum(int(x) * (int(x) - 1) // 2 for x in deg[: g.nU])
                assert side[0] == (0 if wu <= wv else 1)
                for s in (0, 1):                                  # within a side: decreasing
                    ids = order[side == s]                        # degree, ties by id
                    d = deg[ids]
                    assert np.all(d[:-1] >= d[1:])
                    tie = d[:-1] == d[1:]
                    assert np.all(ids[:-1][tie] < ids[1:][tie])


# ----------------------------------------------------------------- duplicates / edges
def test_duplicates_collapse(er1):
    g = er1
    d = synth.with_duplicates(g, seed=77, frac=0.2)
    base = oracle.count(g.nU, g.nV, g.u, g.v)
    c = oracle.count(d.nU, d.nV, d.u, d.v)
    assert c.m == g.m and c.global_count == base.global_count
    np.testing.assert_array_equal(c.per_vertex, base.per_vertex)
    look = {(int(a), int(b)): int(x) for a, b, x in zip(g.u, g.v, base.per_edge)}
    got = [look[(int(a), int(b))] for a, b in zip(d.u, d.v)]
    np.testing.assert_array_equal(c.per_edge, np.array(got, np.uint64))


def test_eq2_sample_matches_ranked_counts(er1):
    g = er1
    c = oracle.count(g.nU, g.nV, g.u, g.v, kind="approx_degree")
    q = np.arange(0, g.m, 37, dtype=np.uint64)
    np.testing.assert_array_equal(oracle.edge_eq2(g.nU, g.nV, g.u, g.v, q), c.per_edge[q.astype(np.int64)])


def test_degenerate_inputs():
    # empty edge list
    c = oracle.count(3, 4, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert c.W == 0 and c.global_count == 0 and c.m == 0 and np.all(c.per_vertex == 0)
    # a star has wedges but no butterflies
    u = np.zeros(10, np.uint32)
    v = np.arange(10, dtype=np.uint32)
    for kind in RANKS:
        c = oracle.count(1, 10, u, v, kind=kind)
        assert c.global_count == 0 and np.all(c.per_edge == 0)
    # ids out of range are rejected
    with pytest.raises(oracle.OracleError):
        oracle.count(2, 2, np.array([2], np.uint32), np.array([0], np.uint32))


# ----------------------------------------------------------------- complement degeneracy
@pytest.mark.parametrize("approx", [False, True])
def test_complement_degeneracy_matches_brute_and_bounds(tiny, approx):
    kind = "approx_complement_degeneracy" if approx else "complement_degeneracy"
    for g in tiny[:25]:
        r = oracle.rank(g.nU, g.nV, g.u, g.v, kind).astype(np.int64)
        np.testing.assert_array_equal(r, brute.complement_degeneracy_rank(g.nU, g.nV, g.u, g.v, approx))
        # the work bound of the paper's proof: for an edge (x, y) with x ranked
        # first, y's neighbours ranked above x number at most deg(x)
        # (2 deg(x) for the approximate order)
        n = g.nU + g.nV
        deg = np.concatenate([np.bincount(g.u, minlength=g.nU), np.bincount(g.v, minlength=g.nV)])
        nb = [[] for _ in range(n)]
        for a, b in set(zip(g.u.tolist(), g.v.tolist())):
            nb[a].append(g.nU + b)
            nb[g.nU + b].append(a)
        for x in range(n):
            for y in nb[x]:
                if r[x] < r[y]:
                    above = sum(1 for z in nb[y] if r[z] > r[x])
                    assert above <= (2 if approx else 1) * deg[x]
        c = oracle.count(g.nU, g.nV, g.u, g.v, kind=kind)
        assert c.W == brute.wedges(g.nU, g.nV, g.u, g.v, r)
        glob, pv, pe = brute.counts(g.nU, g.nV, g.u, g.v)
        assert c.global_count == glob
        np.testing.assert_array_equal(c.per_vertex.astype(np.int64), pv)


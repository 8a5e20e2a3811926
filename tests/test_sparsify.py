"""Approximate counting by sparsification (Sec. "Approximate counting").

CPU: the oracle's estimators are pinned by the probabilities the paper
states (a butterfly survives edge sparsification with probability p^4 and
colourful sparsification with p^3) -- exactly on single butterflies, and as a
sample mean over many seeds on small graphs.  GPU: the device filter keeps
exactly the oracle's edges, and the scaled exact count matches.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import brute
from oracle import sparsify as osp


def test_p_one_keeps_everything():
    g = synth.workload(1)
    for kind in ("edge", "color"):
        u, v, scale = osp.sparsify(g.nU, g.nV, g.u, g.v, kind, 1.0, 7)
        assert u.shape[0] == g.m and scale == 1.0


@pytest.mark.parametrize("kind,p,want", [("edge", 0.5, 0.5 ** 4), ("edge", 0.3, 0.3 ** 4), ("color", 0.5, 0.5 ** 3),
                                         ("color", 0.25, 0.25 ** 3), ("color", 0.3, 0.25 ** 3)])
def test_single_butterfly_survival_probability(kind, p, want):
    """Over many seeds, one K_{2,2} survives with frequency p^4 (edge) or
    ceil(1/p)^-3 (colour: the colours are [1, ceil(1/p)], so p = 0.3 gives 4
    colours and (1/4)^3, the paper's p^3 only when 1/p is an integer)."""
    g = synth.complete_bipartite(2, 2)
    seeds = 20000
    kept = 0
    for s in range(seeds):
        m = osp.keep_mask(2, g.u, g.v, kind, p, 1000 + s)
        kept += int(m.all())
    sd = math.sqrt(want * (1 - want) / seeds)
    assert abs(kept / seeds - want) < 5 * sd
    _, _, scale = osp.sparsify(2, 2, g.u, g.v, kind, p, 1)
    assert scale == pytest.approx(1.0 / want)


@pytest.mark.parametrize("kind,p", [("edge", 0.5), ("color", 0.5), ("color", 0.4)])
def test_estimator_is_unbiased_on_small_graphs(kind, p):
    g = synth.er_graph(0x5A, 30, 40, 500)
    exact = brute.global_count(g.nU, g.nV, g.u, g.v)
    est = []
    for s in range(300):
        u, v, scale = osp.sparsify(g.nU, g.nV, g.u, g.v, kind, p, 77 + s)
        est.append(brute.global_count(g.nU, g.nV, u, v) * scale)
    est = np.array(est)
    assert abs(est.mean() - exact) < 5 * est.std() / math.sqrt(len(est))


@pytest.mark.gpu
def test_gpu_filter_keeps_the_oracle_edges_and_scales():
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    g = synth.chung_lu_graph(0xC0FFEE, 20_000, 60_000, 400_000, 2.1, 2.5, cap_u=3000, cap_v=3000)
    d = synth.with_duplicates(g, seed=9, frac=0.1)
    for kind, p in [("edge", 0.5), ("edge", 0.2), ("color", 0.5), ("color", 0.1), ("color", 0.3)]:
        for seed in (1, 123456789):
            gu, gv = pb.sparsify(d.nU, d.nV, d.u, d.v, kind, p, seed)
            ou, ov, os_ = osp.sparsify(d.nU, d.nV, d.u, d.v, kind, p, seed)
            np.testing.assert_array_equal(gu, ou)
            np.testing.assert_array_equal(gv, ov)
            exact = oracle.count(d.nU, d.nV, ou, ov, per_vertex=False, per_edge=False).global_count
            for agg, rank in [("auto", "degree"), ("hash", "side")]:
                a = pb.approx_global(d.nU, d.nV, d.u, d.v, kind, p, seed, agg=agg, rank=rank)
                assert a.kept_edges == ou.shape[0] and a.kept_count == exact
                assert a.estimate == pytest.approx(exact * os_, rel=1e-15)


@pytest.mark.gpu
def test_gpu_approx_count_with_device_inputs_and_argument_checks():
    import torch
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    g = synth.workload(1)
    du = torch.from_numpy(g.u.view(np.int32)).cuda()
    dv = torch.from_numpy(g.v.view(np.int32)).cuda()
    a = pb.approx_global(g.nU, g.nV, du, dv, "edge", 1.0, 5)   # p = 1 keeps every edge: exact
    assert a.kept_edges == g.m and a.estimate == float(oracle.count(g.nU, g.nV, g.u, g.v).global_count)
    for bad in (0.0, 1.5, -1.0):
        with pytest.raises(pb.PBError) as ei:
            pb.approx_global(g.nU, g.nV, g.u, g.v, "edge", bad, 5)
        assert ei.value.status == 1
    bu = g.u.copy()
    bu[7] = g.nU
    with pytest.raises(pb.PBError) as ei:
        pb.approx_global(g.nU, g.nV, bu, g.v, "edge", 1.0, 5)
    assert ei.value.status == 1

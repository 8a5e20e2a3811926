"""Batched counting (one CUDA-graph launch over many uneven graphs) and the
autotuner: every graph's result in the batch equals its result counted alone
and the oracle's."""
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


def _batch_graphs(k, m_hi=2e5):
    return [synth.batch_graph(i, m_hi=m_hi) for i in range(k)]


def test_batch_equals_alone_and_oracle(pb):
    gs = _batch_graphs(48)
    Gs = [pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree") for g in gs]
    alone = []
    for G in Gs:
        c = G.count_all("auto", edge=False)
        alone.append((c.global_count, c.per_vertex_U.copy(), c.per_vertex_V.copy()))
    B = pb.Batch(Gs, vertex=True)
    assert B.wedges == sum(G.wedges for G in Gs)
    for rep in range(3):                        # replays of the captured graph
        B.run()
        glob = B.globals()
        for i, g in enumerate(gs):
            assert int(glob[i]) == alone[i][0], (i, rep)
            U, V = B.vertex_counts(i)
            np.testing.assert_array_equal(U, alone[i][1])
            np.testing.assert_array_equal(V, alone[i][2])
    for i in range(0, len(gs), 7):
        ref = oracle.count(gs[i].nU, gs[i].nV, gs[i].u, gs[i].v, per_edge=False)
        assert int(glob[i]) == ref.global_count
        np.testing.assert_array_equal(np.concatenate(B.vertex_counts(i)), ref.per_vertex)
    B.free()
    # a batch with one heavy graph among light ones, global counts only
    big = synth.chung_lu_graph(0xC0FFEE, 20_000, 60_000, 400_000, 2.1, 2.5, cap_u=3000, cap_v=3000)
    Gb = pb.Graph.from_edges(big.nU, big.nV, big.u, big.v).rank("approx_degree")
    B = pb.Batch([Gs[0], Gb, Gs[1]], vertex=False)
    B.run()
    ref = oracle.count(big.nU, big.nV, big.u, big.v, per_vertex=False, per_edge=False)
    assert [int(x) for x in B.globals()] == [alone[0][0], ref.global_count, alone[1][0]]
    B.free()
    for G in Gs + [Gb]:
        G.free()


def test_autotune_plan(pb):
    g = synth.workload(1)
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    p = G.autotune()
    du = np.bincount(g.u, minlength=g.nU).astype(np.int64)
    dv = np.bincount(g.v, minlength=g.nV).astype(np.int64)
    w_side = min(int((dv * (dv - 1) // 2).sum()), int((du * (du - 1) // 2).sum()))
    assert p["W_side"] == w_side and p["W_rank"] == G.wedges
    assert abs(p["f_side"] - (w_side - G.wedges) / w_side) < 1e-12
    assert p["rank"] == ("side" if p["f_side"] < 0.1 else "degree")
    assert p["retrieval"] in ("low", "high") and p["agg"] in ("batch", "hash", "hist")
    G.free()

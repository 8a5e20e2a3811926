"""pb_count_noalloc, the entry point for callers that cannot let a library
allocate device memory (a runtime that owns all device memory, or a loop that
must not risk cudaMalloc's implicit synchronisation), against the oracle and
against the regular counting entry point.

Its scratch is a fixed array inside the library, shared by every call, so the
test makes two calls in a row and checks both.  The preprocessed input layout
is built here on the host with numpy from the edge list, independently of the
library's own preprocessing.  The file sorts last so that a run stopping at
the first failure has already run every other test.
"""
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


def preprocessed_layout(nU, nV, u, v):
    """The layout pb_count_noalloc documents, built with numpy: duplicate
    edges removed; ranking by decreasing degree (ties by id); labels U then V,
    each side in rank order; adjacency by decreasing rank; for every entry the
    owner's position in the neighbour's list; per vertex the number of
    neighbours ranked above it."""
    n = nU + nV
    key = np.unique((u.astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64))
    a = (key >> np.uint64(32)).astype(np.int64)
    b = (key & np.uint64(0xFFFFFFFF)).astype(np.int64) + nU
    deg = np.bincount(np.concatenate([a, b]), minlength=n)
    order = np.lexsort((np.arange(n), -deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    label = np.empty(n, np.int64)
    isu = order < nU
    label[order[isu]] = np.arange(nU)
    label[order[~isu]] = nU + np.arange(nV)
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    o = np.lexsort((-rank[dst], label[src]))
    src, dst = src[o], dst[o]
    ls, ld = label[src], label[dst]
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, ls + 1, 1)
    off = np.cumsum(off)
    pos = np.arange(src.shape[0]) - off[ls]
    fwd = ls * n + ld
    srt = np.argsort(fwd)
    rev = srt[np.searchsorted(fwd[srt], ld * n + ls)]
    cpos = pos[rev]
    degp = np.bincount(ls[rank[dst] > rank[src]], minlength=n)
    return n, off, ld, cpos, degp, label


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("which", ["chung_lu", "er"])
def test_noalloc_matches_regular_entry_point_on_two_calls(pb, which):
    import torch
    if which == "chung_lu":
        g = synth.chung_lu_graph(0xC0FFEE, 20_000, 60_000, 400_000, 2.1, 2.5, cap_u=3000, cap_v=3000)
    else:
        g = synth.workload(1)
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    want_global = G.count_global("hist")
    want_U, want_V = G.count_vertex("hist")
    G.free()
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree", per_vertex=True, per_edge=False)
    assert ref.global_count == want_global
    n, off, adj, cpos, degp, label = preprocessed_layout(g.nU, g.nV, g.u, g.v)
    args = [_dev(off), _dev(adj), _dev(cpos), _dev(degp)]
    for _ in range(2):
        out_g = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        out_pv = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        pb.count_noalloc(n, g.nU, *args, out_g, out_pv)
        assert int(out_g.cpu().numpy().view(np.uint64)[0]) == ref.global_count
        pv = out_pv.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(pv[label], ref.per_vertex)          # the oracle, by global id
        np.testing.assert_array_equal(pv[label[: g.nU]], want_U)          # the regular entry point
        np.testing.assert_array_equal(pv[label[g.nU:]], want_V)
        out_g2 = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        pb.count_noalloc(n, g.nU, *args, out_g2)          # global only
        assert int(out_g2.cpu().numpy().view(np.uint64)[0]) == want_global


def test_noalloc_rejects_sides_beyond_its_scratch(pb):
    import torch
    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    o = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(pb.PBError) as ei:
        pb.count_noalloc(40_000_000, 20_000_000, t, t, t, t, o)
    assert ei.value.status == 1
    assert "exceeds the no-allocation scratch" in str(ei.value)


def test_noalloc_on_the_library_layout_and_rejects_a_malformed_one(pb):
    """The layout pb_graph_layout exports is the one pb_count_noalloc takes;
    layouts with a neighbour label out of range, on the wrong side, or a
    deg_x(y) above the degree are rejected with PB_ERR_INVALID (the device
    checks them before using any as an index)."""
    import torch
    g = synth.chung_lu_graph(0xC0FFEE, 20_000, 60_000, 400_000, 2.1, 2.5, cap_u=3000, cap_v=3000)
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree", per_vertex=True, per_edge=False)
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    t = G.layout()
    G.free()
    n = g.nU + g.nV
    out_g = torch.zeros(1, dtype=torch.int64, device="cuda")
    out_pv = torch.zeros(n, dtype=torch.int64, device="cuda")
    pb.count_noalloc(n, g.nU, t["off"], t["adj"], t["cpos"], t["degp"], out_g, out_pv)
    assert int(out_g.cpu().numpy().view(np.uint64)[0]) == ref.global_count
    label = t["label_of"].cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(out_pv.cpu().numpy().view(np.uint64)[label], ref.per_vertex)
    off = t["off"].cpu().numpy().view(np.uint32)
    adj = t["adj"].cpu().numpy().view(np.uint32)
    cpos = t["cpos"].cpu().numpy().view(np.uint32)
    x = int(np.argmax(np.diff(off.astype(np.int64))))     # a vertex with neighbours
    bad_label, wrong_side, big_cpos = adj.copy(), adj.copy(), cpos.copy()
    bad_label[off[x]] = n + 5
    wrong_side[off[x]] = n - 1 if x >= g.nU else 0   # a label on x's own side
    big_cpos[off[x]] = 1 << 30
    for a, c in ((bad_label, cpos), (wrong_side, cpos), (adj, big_cpos)):
        with pytest.raises(pb.PBError) as ei:
            pb.count_noalloc(n, g.nU, t["off"], _dev(a), _dev(c), t["degp"], out_g, out_pv)
        assert ei.value.status == 1 and "malformed layout" in str(ei.value)
    # the shared scratch is usable again after the rejected calls
    pb.count_noalloc(n, g.nU, t["off"], t["adj"], t["cpos"], t["degp"], out_g)
    assert int(out_g.cpu().numpy().view(np.uint64)[0]) == ref.global_count

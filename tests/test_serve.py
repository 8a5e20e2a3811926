"""Serving loop: host-side admission logic (CPU) and, on the GPU, results that
are the same for every request alone and in the concurrent mix."""
import threading
import time

import numpy as np
import pytest

from paper_1907_08607_gb300 import serve


def test_request_stream_is_poisson_with_the_stated_mix():
    reqs, times = serve.request_stream(4000, 100.0, 10, seed=3)
    gaps = np.diff([0.0] + times)
    assert abs(gaps.mean() - 0.01) < 0.01 * 5 / np.sqrt(4000) * 3
    kinds = [r.kind for r in reqs]
    for k, p in (("global", 0.6), ("vertex", 0.3), ("edge", 0.1)):
        frac = kinds.count(k) / len(kinds)
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / len(kinds))
    assert set(r.graph for r in reqs) == set(range(10))


class _FakeGraph:
    """Stands in for a resident graph on the host: records overlap."""
    live = 0
    peak = 0
    mu = threading.Lock()

    def __init__(self, i):
        self.i = i
        self.active = False
        self.wedges = 10

    def count_bytes(self, agg, vertex=True, edge=True, on_device=False):
        return 1000 + (800 if vertex else 0) + (8000 if edge else 0)

    def count_all(self, agg, vertex=True, edge=True, stream=None):
        assert not self.active, "two calls on one graph at once"
        self.active = True
        with _FakeGraph.mu:
            _FakeGraph.live += 1
            _FakeGraph.peak = max(_FakeGraph.peak, _FakeGraph.live)
        time.sleep(0.01)
        with _FakeGraph.mu:
            _FakeGraph.live -= 1
        self.active = False

        class C:
            global_count = self.i
            per_vertex_U = np.full(3, self.i, np.uint64)
            per_vertex_V = np.full(2, self.i, np.uint64)
            per_edge = np.full(4, self.i, np.uint64)
        return C()


def test_admission_overlaps_work_but_never_one_graph_twice(monkeypatch):
    import sys
    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Stream=lambda: None,
                                                                  stream=lambda s: _Null()))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    graphs = [_FakeGraph(i) for i in range(3)]
    srv = serve.Server(graphs, workers=4)
    reqs, _ = serve.request_stream(60, 1000.0, 3, seed=9)
    for r in reqs:
        srv.submit(r)
    done = srv.drain(60, timeout=60)
    srv.close()
    assert len(done) == 60
    assert _FakeGraph.peak >= 2            # different graphs ran at the same time
    assert _FakeGraph.peak <= 3            # never more than one call per graph
    for r in done:
        assert (r.result if r.kind == "global" else r.result[0]) == r.graph


def test_memory_budget_blocks_admission(monkeypatch):
    import sys
    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Stream=lambda: None,
                                                                  stream=lambda s: _Null()))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    _FakeGraph.peak = 0
    graphs = [_FakeGraph(i) for i in range(4)]
    need = serve.predicted_bytes(graphs[0], "edge")
    srv = serve.Server(graphs, workers=4, mem_budget=need)     # room for one request at a time
    reqs = [serve.Request(i, i % 4, "edge") for i in range(12)]
    for r in reqs:
        srv.submit(r)
    srv.drain(12, timeout=60)
    srv.close()
    assert _FakeGraph.peak == 1
    with pytest.raises(ValueError):
        serve.Server(graphs, workers=1, mem_budget=need - 1).submit(serve.Request(99, 0, "edge"))


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


@pytest.mark.gpu
def test_predicted_bytes_bound_the_pool_high_water_mark():
    """The library's bound on a count's allocations (used for admission) is at
    least what the pool's high-water mark rises by during the count, for every
    kind, on graphs from the serving pool and with device or host outputs."""
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    graphs = serve.pool(4, m_lo=1e5, m_hi=3e6)
    for G in graphs:
        for kind in ("global", "vertex", "edge"):
            for on_device in (False, True):
                bound = G.count_bytes("auto", vertex=kind == "vertex", edge=kind == "edge", on_device=on_device)
                used, _ = pb.device_memory(reset_peak=True)
                G.count_all("auto", vertex=kind == "vertex", edge=kind == "edge", on_device=on_device)
                _, peak = pb.device_memory()
                assert peak - used <= bound, (kind, on_device, peak - used, bound)
        G.free()


@pytest.mark.gpu
def test_served_results_equal_alone():
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build
    build.build()
    graphs = serve.pool(6, m_lo=1e4, m_hi=2e6)
    reqs, times = serve.request_stream(60, 200.0, len(graphs), seed=77)
    alone, _ = serve.replay(None, graphs, reqs, times)
    reqs2, _ = serve.request_stream(60, 200.0, len(graphs), seed=77)
    srv = serve.Server(graphs, workers=4)
    served = serve.replay(srv, graphs, reqs2, [0.0] * len(reqs2), timeout=300)[0]   # all at once: maximal overlap
    srv.close()
    assert not [r.error for r in served if r.error]
    assert serve.same_results(alone, served)
    for G in graphs:
        G.free()

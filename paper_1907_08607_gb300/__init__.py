"""Python binding of the GB300 exact butterfly-counting library (libpb.so).

Argument marshalling only: every step of the counting path runs in the CUDA
kernels behind the C ABI of ``include/pb.h``.  PyTorch supplies device memory
and the current CUDA stream.  There is no CPU fallback: if ``libpb.so`` has
not been built (``paper_1907_08607_gb300.build.build()``) or no CUDA device is
present, calls raise.

Names follow the paper (Shi & Shun, "Parallel Algorithms for Butterfly
Computations"): ranking ``side`` / ``degree`` / ``approx_degree`` (Sec.
"Ranking"), wedge aggregation ``sort`` / ``hash`` / ``hist`` / ``batch``
(Sec. "Wedge aggregation"), global / per-vertex / per-edge counts
(Algorithms 3 and 4).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpb.so")

RANKS = {"side": 0, "degree": 1, "approx_degree": 2, "complement_degeneracy": 3,
         "approx_complement_degeneracy": 4}
AGGS = {"sort": 0, "hash": 1, "hist": 2, "batch": 3, "auto": 4}
RETRIEVALS = {"low": 0, "high": 1, "auto": 2}
BUTTERFLY_AGGS = {"atomic": 0, "sort": 1}
STATUS = {0: "PB_OK", 1: "PB_ERR_INVALID", 2: "PB_ERR_NOMEM", 3: "PB_ERR_CUDA", 4: "PB_ERR_SCRATCH",
          5: "PB_ERR_TIMEOUT", 6: "PB_ERR_OVERFLOW"}

# Every function the C ABI exports (include/pb.h).
ABI_SYMBOLS = ["pb_graph_from_edges", "pb_rank", "pb_rank_custom", "pb_graph_ranks", "pb_count_global",
               "pb_count_vertex", "pb_count_edge", "pb_count_all", "pb_wedge_count", "pb_graph_info",
               "pb_graph_free", "pb_kernel_launches", "pb_last_error", "pb_status_string",
               "pb_profile_enable", "pb_profile_reset", "pb_profile_read", "pb_count_noalloc",
               "pb_set_retrieval", "pb_count_owner_range", "pb_wedge_prefix", "pb_sparsify", "pb_autotune",
               "pb_batch_create", "pb_batch_run", "pb_batch_globals", "pb_batch_vertex", "pb_batch_wedges",
               "pb_batch_free", "pb_set_butterfly_aggregation", "pb_count_approx", "pb_graph_layout",
               "pb_calibrate_atomics", "pb_set_plan", "pb_count_bytes", "pb_set_grid_share",
               "pb_device_memory"]

PHASES = ["build", "rank", "classify", "light", "medium", "heavy", "sort", "output", "large"]

_lock = threading.Lock()
_lib = None


class PBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [("nU", ctypes.c_uint32), ("nV", ctypes.c_uint32), ("m_in", ctypes.c_uint64),
                ("m", ctypes.c_uint64), ("max_deg_U", ctypes.c_uint32), ("max_deg_V", ctypes.c_uint32),
                ("rank_kind", ctypes.c_int32), ("W", ctypes.c_uint64), ("max_wedges_x1", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64)]


class Plan(ctypes.Structure):
    _fields_ = [("rank_kind", ctypes.c_int32), ("retrieval", ctypes.c_int32), ("agg", ctypes.c_int32),
                ("hub_cluster", ctypes.c_uint32), ("hub_min", ctypes.c_uint64), ("f_side", ctypes.c_double),
                ("W_side", ctypes.c_uint64), ("W_rank", ctypes.c_uint64), ("max_owner_wedges", ctypes.c_uint64),
                ("light_max", ctypes.c_uint32), ("med_max", ctypes.c_uint32), ("large_max", ctypes.c_uint32),
                ("hot", ctypes.c_uint32), ("heavy_slots", ctypes.c_uint32), ("hot_hit", ctypes.c_double),
                ("owners", ctypes.c_uint64 * 4), ("wedges", ctypes.c_uint64 * 4), ("slot_bytes", ctypes.c_uint64), ("slot_bytes_dense", ctypes.c_uint64),
                ("slot_bytes_hash", ctypes.c_uint64), ("resident_blocks", ctypes.c_uint32),
                ("mid_segment", ctypes.c_double), ("scratch_bytes", ctypes.c_uint64)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 9), ("launches", ctypes.c_uint64 * 9),
                ("wedges", ctypes.c_uint64 * 9), ("records", ctypes.c_uint64 * 9)]

    def as_dict(self):
        return {ph: dict(ms=self.ms[i], launches=int(self.launches[i]), wedges=int(self.wedges[i]),
                         records=int(self.records[i])) for i, ph in enumerate(PHASES)}


def load_library(path: str = LIB_PATH):
    """Load libpb.so and declare the C signatures (no compute)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libpb.so not built at {path}; run paper_1907_08607_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.pb_graph_from_edges.argtypes = [u32, u32, u64, vp, vp, i32, vp, ctypes.POINTER(vp)]
        lib.pb_rank.argtypes = [vp, i32, vp]
        lib.pb_rank_custom.argtypes = [vp, vp, i32, vp]
        lib.pb_graph_ranks.argtypes = [vp, vp, i32, vp]
        lib.pb_count_global.argtypes = [vp, i32, u64, u64p, vp]
        lib.pb_count_vertex.argtypes = [vp, i32, u64, vp, vp, i32, vp]
        lib.pb_count_edge.argtypes = [vp, i32, u64, vp, i32, vp]
        lib.pb_count_all.argtypes = [vp, i32, u64, u64p, vp, vp, vp, i32, vp]
        lib.pb_wedge_count.argtypes = [vp, u64p]
        lib.pb_graph_info.argtypes = [vp, ctypes.POINTER(GraphInfo)]
        lib.pb_graph_free.argtypes = [vp]
        for f in ("pb_graph_from_edges", "pb_rank", "pb_rank_custom", "pb_graph_ranks", "pb_count_global",
                  "pb_count_vertex", "pb_count_edge", "pb_count_all", "pb_wedge_count", "pb_graph_info",
                  "pb_graph_free"):
            getattr(lib, f).restype = i32
        lib.pb_kernel_launches.argtypes = []
        lib.pb_kernel_launches.restype = ctypes.c_uint64
        lib.pb_last_error.argtypes = []
        lib.pb_last_error.restype = ctypes.c_char_p
        lib.pb_status_string.argtypes = [i32]
        lib.pb_status_string.restype = ctypes.c_char_p
        lib.pb_profile_enable.argtypes = [i32]
        lib.pb_profile_enable.restype = None
        lib.pb_profile_reset.argtypes = []
        lib.pb_profile_reset.restype = None
        lib.pb_profile_read.argtypes = [ctypes.POINTER(Profile)]
        lib.pb_profile_read.restype = i32
        lib.pb_count_noalloc.argtypes = [u64, u32, vp, vp, vp, vp, vp, vp, vp]
        lib.pb_count_noalloc.restype = i32
        lib.pb_set_retrieval.argtypes = [vp, i32]
        lib.pb_set_retrieval.restype = i32
        lib.pb_set_butterfly_aggregation.argtypes = [vp, i32]
        lib.pb_set_butterfly_aggregation.restype = i32
        lib.pb_count_owner_range.argtypes = [vp, i32, u64, u32, u32, u64p, vp, vp, vp, i32, vp]
        lib.pb_count_owner_range.restype = i32
        lib.pb_wedge_prefix.argtypes = [vp, vp, i32, vp]
        lib.pb_wedge_prefix.restype = i32
        lib.pb_sparsify.argtypes = [u32, u32, u64, vp, vp, i32, i32, ctypes.c_double, u64, vp, vp, u64p, vp]
        lib.pb_sparsify.restype = i32
        lib.pb_count_approx.argtypes = [u32, u32, u64, vp, vp, i32, i32, ctypes.c_double, u64, i32, i32, u64,
                                         ctypes.POINTER(ctypes.c_double), u64p, u64p, vp]
        lib.pb_count_approx.restype = i32
        lib.pb_calibrate_atomics.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
        lib.pb_calibrate_atomics.restype = i32
        lib.pb_graph_layout.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
        lib.pb_graph_layout.restype = i32
        lib.pb_autotune.argtypes = [vp, u64, ctypes.POINTER(Plan)]
        lib.pb_count_bytes.argtypes = [vp, i32, u64, i32, i32, i32, u64p]
        lib.pb_count_bytes.restype = i32
        lib.pb_set_grid_share.argtypes = [vp, ctypes.c_double]
        lib.pb_set_grid_share.restype = i32
        lib.pb_device_memory.argtypes = [i32, u64p, u64p]
        lib.pb_device_memory.restype = i32
        lib.pb_set_plan.argtypes = [vp, ctypes.POINTER(Plan)]
        lib.pb_set_plan.restype = i32
        lib.pb_batch_create.argtypes = [ctypes.POINTER(vp), u32, i32, u64, vp, ctypes.POINTER(vp)]
        lib.pb_batch_run.argtypes = [vp, vp]
        lib.pb_batch_globals.argtypes = [vp, u64p, vp]
        lib.pb_batch_vertex.argtypes = [vp, u32, vp, vp, i32, vp]
        lib.pb_batch_wedges.argtypes = [vp, u64p]
        lib.pb_batch_free.argtypes = [vp]
        for f in ("pb_autotune", "pb_batch_create", "pb_batch_run", "pb_batch_globals", "pb_batch_vertex",
                  "pb_batch_wedges", "pb_batch_free"):
            getattr(lib, f).restype = i32
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = _lib.pb_last_error().decode(errors="replace") if _lib else ""
        raise PBError(rc, msg)


def kernel_launches() -> int:
    return int(load_library().pb_kernel_launches())


def profile(enable: bool | None = None, reset: bool = False) -> dict:
    """Per-phase device time / launches / wedges recorded by the library
    (CUDA events on the calling stream), optionally toggling recording."""
    lib = load_library()
    if reset:
        lib.pb_profile_reset()
    if enable is not None:
        lib.pb_profile_enable(int(enable))
    p = Profile()
    _check(lib.pb_profile_read(ctypes.byref(p)))
    return p.as_dict()


def calibrate_atomics(scattered: bool = False, stream=None) -> float:
    """64-bit L2 atomic-add throughput of the current device, operations/s
    (pb_calibrate_atomics): coalesced (per-edge pattern) or scattered."""
    out = ctypes.c_double()
    _check(load_library().pb_calibrate_atomics(int(scattered), ctypes.byref(out), _stream(stream)))
    return out.value


def device_memory(reset_peak: bool = False) -> tuple[int, int]:
    """(bytes in use, high-water mark) of the library's device memory pool."""
    used, peak = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().pb_device_memory(int(reset_peak), ctypes.byref(used), ctypes.byref(peak)))
    return int(used.value), int(peak.value)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the butterfly library runs on the GPU only")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _edge_arg(x, torch):
    """(pointer, on_device, keepalive) for a uint32 edge array (torch or numpy)."""
    if isinstance(x, torch.Tensor):
        if x.dtype not in (torch.int32, torch.uint32):
            raise TypeError("edge tensors must be int32/uint32")
        if not x.is_contiguous():
            x = x.contiguous()
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=np.uint32)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def count_noalloc(n: int, nU: int, off, adj, cpos, degp, out_global, out_pv=None, stream=None) -> None:
    """pb_count_noalloc: counts on an already preprocessed graph held in
    caller-owned device tensors, with no device allocation by the library (for
    callers whose runtime owns all device memory).  Inputs are int32/uint32
    CUDA tensors in the layout of include/pb.h; out_global is a 1-element and
    out_pv an n-element int64 CUDA tensor (uint64 bit patterns)."""
    lib = load_library()
    for t in (off, adj, cpos, degp, out_global) + ((out_pv,) if out_pv is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("pb_count_noalloc takes contiguous CUDA tensors")
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    _check(lib.pb_count_noalloc(n, nU, p(off), p(adj), p(cpos), p(degp), p(out_global), p(out_pv),
                                _stream(stream)))


SPARSIFY = {"edge": 0, "color": 1}


def sparsify(nU: int, nV: int, u, v, kind: str, p: float, seed: int, stream=None):
    """Kept edge pairs (host uint32 arrays, input order) of edge or colourful
    sparsification (pb_sparsify)."""
    lib = load_library()
    torch = _torch()
    pu, du, ku = _edge_arg(u, torch)
    pv, dv, kv = _edge_arg(v, torch)
    if du:
        raise ValueError("pass host arrays")
    m = int(ku.shape[0])
    ou = np.empty(max(m, 1), np.uint32)
    ov = np.empty(max(m, 1), np.uint32)
    om = ctypes.c_uint64()
    _check(lib.pb_sparsify(nU, nV, m, pu, pv, 0, SPARSIFY[kind], p, seed, ctypes.c_void_p(ou.ctypes.data),
                           ctypes.c_void_p(ov.ctypes.data), ctypes.byref(om), _stream(stream)))
    k = int(om.value)
    return ou[:k].copy(), ov[:k].copy()


@dataclass
class Approx:
    estimate: float
    kept_count: int
    kept_edges: int


def approx_global(nU: int, nV: int, u, v, kind: str = "edge", p: float = 0.5, seed: int = 1,
                  agg: str = "auto", rank: str = "degree", scratch_bytes: int = 0, stream=None) -> Approx:
    """pb_count_approx: approximate total butterfly count (Sec. "Approximate
    counting"); sparsification, exact count of the kept graph and scaling all
    run in the library."""
    lib = load_library()
    torch = _torch()
    pu, du, ku = _edge_arg(u, torch)
    pv, dv, kv = _edge_arg(v, torch)
    if du != dv:
        raise ValueError("u and v must both be on the device or both on the host")
    est, kc, ke = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.pb_count_approx(nU, nV, int(ku.shape[0]), pu, pv, du, SPARSIFY[kind], p, seed, RANKS[rank],
                               AGGS[agg], scratch_bytes, ctypes.byref(est), ctypes.byref(kc), ctypes.byref(ke),
                               _stream(stream)))
    return Approx(est.value, int(kc.value), int(ke.value))


@dataclass
class Counts:
    global_count: int | None
    per_vertex_U: object | None
    per_vertex_V: object | None
    per_edge: object | None


class Graph:
    """A bipartite graph resident on the current CUDA device."""

    def __init__(self, handle: ctypes.c_void_p, nU: int, nV: int, m_in: int):
        self._h = handle
        self.nU, self.nV, self.m_in = nU, nV, m_in

    # -- construction ---------------------------------------------------
    @classmethod
    def from_edges(cls, nU: int, nV: int, u, v, stream=None) -> "Graph":
        lib = load_library()
        torch = _torch()
        pu, du, ku = _edge_arg(u, torch)
        pv, dv, kv = _edge_arg(v, torch)
        if du != dv:
            raise ValueError("u and v must both be on the device or both on the host")
        m = int(ku.shape[0])
        if int(kv.shape[0]) != m:
            raise ValueError("u and v differ in length")
        h = ctypes.c_void_p()
        _check(lib.pb_graph_from_edges(nU, nV, m, pu, pv, du, _stream(stream), ctypes.byref(h)))
        return cls(h, nU, nV, m)

    def free(self):
        if self._h:
            load_library().pb_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    # -- PREPROCESS -----------------------------------------------------
    def rank(self, kind: str = "degree", stream=None) -> "Graph":
        _check(load_library().pb_rank(self._h, RANKS[kind], _stream(stream)))
        return self

    def rank_custom(self, rank_of, stream=None) -> "Graph":
        torch = _torch()
        p, dev, keep = _edge_arg(rank_of, torch)
        _check(load_library().pb_rank_custom(self._h, p, dev, _stream(stream)))
        return self

    def set_retrieval(self, which: str = "auto") -> "Graph":
        """Wedge owner for later counts: "low" (Algorithm 2), "high" (the
        cache optimisation) or "auto"."""
        _check(load_library().pb_set_retrieval(self._h, RETRIEVALS[which]))
        return self

    def set_butterfly_aggregation(self, which: str = "atomic") -> "Graph":
        """How per-vertex / per-edge contributions reach their counters:
        "atomic" adds, or "sort" re-aggregation (needs agg="sort")."""
        _check(load_library().pb_set_butterfly_aggregation(self._h, BUTTERFLY_AGGS[which]))
        return self

    def autotune(self, scratch_bytes: int = 0) -> dict:
        """The autotuner's plan for this graph and scratch budget (pb_autotune)."""
        p = Plan()
        _check(load_library().pb_autotune(self._h, scratch_bytes, ctypes.byref(p)))
        inv_rank = {v: k for k, v in RANKS.items()}
        inv_rt = {v: k for k, v in RETRIEVALS.items()}
        inv_agg = {v: k for k, v in AGGS.items()}
        return dict(rank=inv_rank.get(p.rank_kind), retrieval=inv_rt.get(p.retrieval), agg=inv_agg.get(p.agg),
                    hub_cluster=p.hub_cluster, hub_min=p.hub_min, f_side=p.f_side, W_side=p.W_side, W_rank=p.W_rank,
                    max_owner_wedges=p.max_owner_wedges, light_max=p.light_max, med_max=p.med_max,
                    large_max=p.large_max, hot=p.hot,
                    heavy_slots=p.heavy_slots, hot_hit=p.hot_hit, owners=list(p.owners), wedges=list(p.wedges),
                    slot_bytes=p.slot_bytes, slot_bytes_dense=p.slot_bytes_dense, slot_bytes_hash=p.slot_bytes_hash,
                    resident_blocks=p.resident_blocks, mid_segment=p.mid_segment, scratch_bytes=p.scratch_bytes)

    def count_bytes(self, agg: str = "auto", scratch_bytes: int = 0, vertex: bool = True, edge: bool = True,
                    on_device: bool = False) -> int:
        """Upper bound on the device memory such a count allocates (pb_count_bytes)."""
        out = ctypes.c_uint64()
        _check(load_library().pb_count_bytes(self._h, AGGS[agg], scratch_bytes, int(vertex), int(edge),
                                             int(on_device), ctypes.byref(out)))
        return int(out.value)

    def set_grid_share(self, share: float) -> "Graph":
        """Share of the device's resident blocks later counts take (pb_set_grid_share)."""
        _check(load_library().pb_set_grid_share(self._h, share))
        return self

    def set_plan(self, plan: dict | None) -> "Graph":
        """Pins a plan (a dict as autotune() returns, fields may be changed)
        for later "auto" counts; None returns to planning per count."""
        lib = load_library()
        if plan is None:
            _check(lib.pb_set_plan(self._h, None))
            return self
        p = Plan()
        p.rank_kind = RANKS.get(plan.get("rank") or "degree", 1)
        p.retrieval = RETRIEVALS[plan["retrieval"]]
        p.agg = AGGS[plan["agg"]]
        p.hub_cluster = plan.get("hub_cluster", 1)
        p.hub_min = plan.get("hub_min", 2 ** 64 - 1)
        p.light_max = plan.get("light_max", 768)
        p.med_max = plan.get("med_max", 4096)
        p.large_max = plan.get("large_max", 4096)
        p.hot = plan.get("hot", 16384)
        _check(lib.pb_set_plan(self._h, ctypes.byref(p)))
        return self

    def layout(self, stream=None) -> dict:
        """The PREPROCESS output as int32 CUDA tensors (uint32 bit patterns):
        off, adj, cpos, degp (the input of count_noalloc) and label_of."""
        torch = _torch()
        n, na = self.nU + self.nV, 2 * self.info().m
        t = {k: torch.empty(c, dtype=torch.int32, device="cuda") for k, c in
             (("off", n + 1), ("adj", max(na, 1)), ("cpos", max(na, 1)), ("degp", n), ("label_of", n))}
        p = lambda k: ctypes.c_void_p(t[k].data_ptr())  # noqa: E731
        _check(load_library().pb_graph_layout(self._h, p("off"), p("adj"), p("cpos"), p("degp"), p("label_of"), 1,
                                              _stream(stream)))
        return t

    def ranks(self, stream=None) -> np.ndarray:
        out = np.empty(self.nU + self.nV, np.uint32)
        _check(load_library().pb_graph_ranks(self._h, ctypes.c_void_p(out.ctypes.data), 0, _stream(stream)))
        return out

    @property
    def wedges(self) -> int:
        W = ctypes.c_uint64()
        _check(load_library().pb_wedge_count(self._h, ctypes.byref(W)))
        return int(W.value)

    def info(self) -> GraphInfo:
        inf = GraphInfo()
        _check(load_library().pb_graph_info(self._h, ctypes.byref(inf)))
        return inf

    # -- counting -------------------------------------------------------
    def count_global(self, agg: str = "auto", scratch_bytes: int = 0, stream=None) -> int:
        out = ctypes.c_uint64()
        _check(load_library().pb_count_global(self._h, AGGS[agg], scratch_bytes, ctypes.byref(out),
                                              _stream(stream)))
        return int(out.value)

    def count_vertex(self, agg: str = "auto", scratch_bytes: int = 0, on_device: bool = False, stream=None):
        c = self.count_all(agg, scratch_bytes, glob=False, vertex=True, edge=False, on_device=on_device,
                           stream=stream)
        return c.per_vertex_U, c.per_vertex_V

    def count_edge(self, agg: str = "auto", scratch_bytes: int = 0, on_device: bool = False, stream=None):
        return self.count_all(agg, scratch_bytes, glob=False, vertex=False, edge=True, on_device=on_device,
                              stream=stream).per_edge

    def wedge_prefix(self, stream=None) -> np.ndarray:
        """Per-owner exclusive wedge prefix (n + 1 uint64) under the current
        retrieval; the last entry is W."""
        out = np.empty(self.nU + self.nV + 1, np.uint64)
        _check(load_library().pb_wedge_prefix(self._h, ctypes.c_void_p(out.ctypes.data), 0, _stream(stream)))
        return out

    def count_all(self, agg: str = "auto", scratch_bytes: int = 0, glob: bool = True, vertex: bool = True,
                  edge: bool = True, on_device: bool = False, out=None, stream=None,
                  owners: tuple[int, int] | None = None) -> Counts:
        """One wedge pass producing any of the three outputs.  Host outputs are
        uint64 numpy arrays; device outputs are int64 CUDA tensors holding the
        uint64 bit patterns (``out`` may pass preallocated ones as a dict)."""
        lib = load_library()
        torch = _torch()
        g = ctypes.c_uint64() if glob else None
        U = V = E = None
        if on_device:
            out = out or {}
            if vertex:
                U = out.get("U", torch.empty(self.nU, dtype=torch.int64, device="cuda"))
                V = out.get("V", torch.empty(self.nV, dtype=torch.int64, device="cuda"))
            if edge:
                E = out.get("E", torch.empty(self.m_in, dtype=torch.int64, device="cuda"))
            ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        else:
            out = out or {}
            if vertex:
                U = out.get("U", np.empty(self.nU, np.uint64))
                V = out.get("V", np.empty(self.nV, np.uint64))
            if edge:
                E = out.get("E", np.empty(self.m_in, np.uint64))

            def ptr(a):
                if a is None:
                    return None
                if isinstance(a, torch.Tensor):   # e.g. pinned host buffers
                    return ctypes.c_void_p(a.data_ptr())
                return ctypes.c_void_p(a.ctypes.data)
        if owners is None:
            _check(lib.pb_count_all(self._h, AGGS[agg], scratch_bytes, ctypes.byref(g) if g is not None else None,
                                    ptr(U), ptr(V), ptr(E), int(on_device), _stream(stream)))
        else:
            _check(lib.pb_count_owner_range(self._h, AGGS[agg], scratch_bytes, int(owners[0]), int(owners[1]),
                                            ctypes.byref(g) if g is not None else None, ptr(U), ptr(V), ptr(E),
                                            int(on_device), _stream(stream)))
        return Counts(int(g.value) if g is not None else None, U, V, E)


class Batch:
    """Many ranked graphs counted together: one persistent kernel per work
    tier over all their owners, captured once in a CUDA graph and replayed
    by run()."""

    def __init__(self, graphs, vertex: bool = True, scratch_bytes: int = 0, stream=None):
        lib = load_library()
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g._h for g in self.graphs])
        h = ctypes.c_void_p()
        _check(lib.pb_batch_create(arr, len(self.graphs), int(vertex), scratch_bytes, _stream(stream),
                                   ctypes.byref(h)))
        self._h = h
        self.vertex = vertex

    def run(self, stream=None):
        _check(load_library().pb_batch_run(self._h, _stream(stream)))

    def globals(self, stream=None) -> np.ndarray:
        out = np.empty(len(self.graphs), np.uint64)
        _check(load_library().pb_batch_globals(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                               _stream(stream)))
        return out

    def vertex_counts(self, i: int, stream=None):
        g = self.graphs[i]
        U = np.empty(g.nU, np.uint64)
        V = np.empty(g.nV, np.uint64)
        _check(load_library().pb_batch_vertex(self._h, i, ctypes.c_void_p(U.ctypes.data),
                                              ctypes.c_void_p(V.ctypes.data), 0, _stream(stream)))
        return U, V

    @property
    def wedges(self) -> int:
        W = ctypes.c_uint64()
        _check(load_library().pb_batch_wedges(self._h, ctypes.byref(W)))
        return int(W.value)

    def free(self):
        if getattr(self, "_h", None):
            load_library().pb_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


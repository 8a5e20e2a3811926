"""Seeded synthetic bipartite graphs (input generation only).

Nothing here counts wedges or butterflies: the module draws edge lists that
both the CPU oracle and the CUDA library consume.  The heavy lifting is in
``synth.c`` (counter-based SplitMix64 draws, Vose alias tables, first-occurrence
deduplication), compiled on first use with gcc.

Workload recipes (stand-ins for the KONECT graphs of the paper's Table 1,
which are not available):

* ``er_graph``        - uniform distinct pairs (bipartite Erdos-Renyi).
* ``chung_lu_graph``  - expected degrees w_i = min(cap, c (i+1)^(-1/(gamma-1)))
  with c fixed so that sum w = m; endpoints drawn proportional to w, duplicate
  pairs rejected; ids then randomly permuted within each side so that id order
  carries no degree information.
* ``workload(i)``     - the named configurations (ER 2k x 3k, Chung-Lu 1M x 4M,
  Chung-Lu 20M x 60M) and the per-graph recipe of the 1,024-graph batch.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 0x9B7F0000


def build() -> str:
    """Compile synth.c into _build/libsynth.so (idempotent)."""
    src = os.path.join(_HERE, "synth.c")
    os.makedirs(_BUILD, exist_ok=True)
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.synth_er.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_int, u32p, u32p]
            lib.synth_er.restype = ctypes.c_int
            lib.synth_chung_lu.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, u32p, u32p]
            lib.synth_chung_lu.restype = ctypes.c_int
            lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_draw.restype = ctypes.c_uint64
            lib.synth_shuffle_pairs.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.synth_shuffle_pairs.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclass
class Graph:
    """A bipartite edge list: u[k] in [0, nU), v[k] in [0, nV)."""
    nU: int
    nV: int
    u: np.ndarray
    v: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.u.shape[0])


def er_graph(seed: int, nU: int, nV: int, m: int, name: str = "") -> Graph:
    lib = _load()
    u = np.empty(m, np.uint32)
    v = np.empty(m, np.uint32)
    rc = lib.synth_er(seed, nU, nV, m, _threads(), _ptr(u), _ptr(v))
    if rc != 0:
        raise ValueError(f"synth_er failed ({rc}) for nU={nU} nV={nV} m={m}")
    return Graph(nU, nV, u, v, name or f"er_{nU}x{nV}_m{m}")


def chung_lu_graph(seed: int, nU: int, nV: int, m: int, gamma_u: float, gamma_v: float,
                   cap_u: float = 1e5, cap_v: float = 1e5, permute: bool = True,
                   name: str = "") -> Graph:
    lib = _load()
    u = np.empty(m, np.uint32)
    v = np.empty(m, np.uint32)
    rc = lib.synth_chung_lu(seed, nU, nV, m, gamma_u, gamma_v, cap_u, cap_v, int(permute),
                            _threads(), _ptr(u), _ptr(v))
    if rc != 0:
        raise ValueError(f"synth_chung_lu failed ({rc}) for nU={nU} nV={nV} m={m}")
    return Graph(nU, nV, u, v, name or f"cl_{nU}x{nV}_m{m}")


def draw(seed: int, stream: int, k: int) -> int:
    """The k-th 64-bit draw of sub-stream `stream` of `seed`."""
    return int(_load().synth_draw(seed, stream, k))


def uniform(seed: int, stream: int, k: int) -> float:
    return (draw(seed, stream, k) >> 11) * (1.0 / 9007199254740992.0)


def with_duplicates(g: Graph, seed: int, frac: float = 0.1) -> Graph:
    """The same edge set with a seeded fraction of edges repeated and the list
    shuffled: an input with duplicate pairs in arbitrary order."""
    rep = int(g.m * frac)
    u = np.concatenate([g.u, g.u[:rep]])
    v = np.concatenate([g.v, g.v[:rep]])
    _load().synth_shuffle_pairs(seed, u.shape[0], _ptr(u), _ptr(v))
    return Graph(g.nU, g.nV, u, v, g.name + "_dup")


def complete_bipartite(a: int, b: int) -> Graph:
    uu, vv = np.meshgrid(np.arange(a, dtype=np.uint32), np.arange(b, dtype=np.uint32),
                         indexing="ij")
    return Graph(a, b, uu.ravel().copy(), vv.ravel().copy(), f"K{a},{b}")


# ---------------------------------------------------------------------------
# Named workloads.

WORKLOADS = {
    1: "ER |U|=2000 |V|=3000 m=20000",
    2: "Chung-Lu |U|=1M |V|=4M m=50M gamma 2.1/2.5 cap 1e5",
    3: "Chung-Lu |U|=20M |V|=60M m=300M gamma 2.0/2.0 cap 1e5",
}


def workload(idx: int) -> Graph:
    seed = SEED_BASE + idx
    if idx == 1:
        return er_graph(seed, 2000, 3000, 20000, name="er_2000x3000_m2e4")
    if idx == 2:
        return chung_lu_graph(seed, 1_000_000, 4_000_000, 50_000_000, 2.1, 2.5,
                              name="cl_1Mx4M_m5e7")
    if idx == 3:
        return chung_lu_graph(seed, 20_000_000, 60_000_000, 300_000_000, 2.0, 2.0,
                              name="cl_20Mx60M_m3e8")
    if idx == -2:  # quarter-scale copy of workload 2 (profiling)
        return chung_lu_graph(seed, 250_000, 1_000_000, 12_500_000, 2.1, 2.5,
                              name="cl_250kx1M_m1.25e7")
    if idx == -3:  # 1/16-scale copy of workload 3 (profiling)
        return chung_lu_graph(seed, 1_250_000, 3_750_000, 18_750_000, 2.0, 2.0,
                              name="cl_1.25Mx3.75M_m1.875e7")
    raise KeyError(idx)


def batch_graph_params(i: int, seed: int = SEED_BASE + 4, m_lo: float = 1e3,
                       m_hi: float = 1e6) -> dict:
    """Parameters of graph i of the batched workload: m log-uniform in
    [m_lo, m_hi], Erdos-Renyi or Chung-Lu by coin flip (gamma uniform in
    [1.8, 2.8]), |V|/|U| log-uniform in [0.1, 10], |U| = ceil(sqrt(m / (ratio *
    0.01))) clamped so that |U| |V| >= 4 m."""
    gseed = draw(seed, 100, i)
    m = int(round(math.exp(math.log(m_lo) + uniform(gseed, 1, 0) * (math.log(m_hi) - math.log(m_lo)))))
    ratio = math.exp(math.log(0.1) + uniform(gseed, 1, 1) * (math.log(10.0) - math.log(0.1)))
    nU = max(2, math.ceil(math.sqrt(m / (ratio * 0.01))))
    nV = max(2, math.ceil(ratio * nU))
    while nU * nV < 4 * m:
        nU += 1
        nV = max(2, math.ceil(ratio * nU))
    cl = uniform(gseed, 1, 2) < 0.5
    gamma = 1.8 + uniform(gseed, 1, 3) * 1.0
    return dict(seed=gseed, m=m, nU=nU, nV=nV, chung_lu=cl, gamma=gamma)


def batch_graph(i: int, **kw) -> Graph:
    p = batch_graph_params(i, **kw)
    if p["chung_lu"]:
        return chung_lu_graph(p["seed"], p["nU"], p["nV"], p["m"], p["gamma"], p["gamma"],
                              cap_u=max(1.0, min(1e5, p["nV"] / 2)),
                              cap_v=max(1.0, min(1e5, p["nU"] / 2)), name=f"batch{i}_cl")
    return er_graph(p["seed"], p["nU"], p["nV"], p["m"], name=f"batch{i}_er")

"""TEST INFRASTRUCTURE ONLY -- the CPU oracle for exact butterfly counting.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_1907_08607_gb300``) and never imports it.

Two independent forms:

* ``count`` / ``rank`` / ``wedges`` / ``edge_eq2`` -- ``pb_oracle.c``, plain
  C following the paper's steps in order (dedupe; PREPROCESS, Algorithm 1;
  GET-WEDGES, Algorithm 2; dense-array aggregation, the paper's simple batching;
  Algorithms 3 and 4 with atomic adds), plus Eq. 2 evaluated edge by edge.
* ``brute`` -- the definitions themselves (butterfly definition in the
  preliminaries, Eq. 1 and Eq. 2 of the counting lemma) over all vertex pairs,
  for tiny graphs.

Every function here is pinned by ``tests/test_oracle_*.py`` against the paper's
worked example (Figs. 1-2), closed forms on complete bipartite graphs, brute
force, and counting invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

from . import brute  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpboracle.so")
_lock = threading.Lock()
_lib = None

RANK_SIDE, RANK_DEGREE, RANK_APPROX_DEGREE, RANK_CODEGEN, RANK_APPROX_CODEGEN = 0, 1, 2, 3, 4
RANK_KINDS = {"side": RANK_SIDE, "degree": RANK_DEGREE, "approx_degree": RANK_APPROX_DEGREE,
              "complement_degeneracy": RANK_CODEGEN, "approx_complement_degeneracy": RANK_APPROX_CODEGEN}


class OracleError(RuntimeError):
    pass


def build() -> str:
    """Compile pb_oracle.c into _build/libpboracle.so (idempotent)."""
    src = os.path.join(_HERE, "pb_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.orc_rank.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p,
                                     ctypes.c_int, u32p]
            lib.orc_count.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p,
                                      ctypes.c_int, u32p, ctypes.c_int, u64p, u64p, u64p, u64p, u64p]
            lib.orc_wedges.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p,
                                       ctypes.c_int, u32p, u64p]
            lib.orc_edge_eq2.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p,
                                         u32p, ctypes.c_uint64, u64p, ctypes.c_int, u64p]
            lib.orc_count_range.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p,
                                            ctypes.c_int, u32p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                            u64p, u64p, u64p, u64p, u64p]
            lib.orc_owner_wedges.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p,
                                             ctypes.c_int, u32p, u64p]
            lib.orc_count_range.restype = ctypes.c_int
            lib.orc_owner_wedges.restype = ctypes.c_int
            lib.orc_vertex_eq1.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p,
                                           u32p, ctypes.c_uint64, u64p, u64p]
            for f in (lib.orc_rank, lib.orc_count, lib.orc_wedges, lib.orc_edge_eq2, lib.orc_vertex_eq1):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def threads() -> int:
    return max(1, os.cpu_count() or 1)


@dataclass
class Counts:
    nU: int
    W: int                  # retrieved wedges under the ranking used
    global_count: int
    m: int                  # distinct edges
    per_vertex: np.ndarray | None   # uint64 [nU + nV], U ids then V ids
    per_edge: np.ndarray | None     # uint64 [m_in], input order


def rank(nU: int, nV: int, u, v, kind: str | int) -> np.ndarray:
    """rank[id] (U ids then V ids) under the paper's ranking `kind`."""
    lib = _load()
    k = RANK_KINDS[kind] if isinstance(kind, str) else int(kind)
    u, pu = _u32(u)
    v, pv = _u32(v)
    out = np.empty(nU + nV, np.uint32)
    _check(lib.orc_rank(nU, nV, u.shape[0], pu, pv, k, _u32(out)[1]), "orc_rank")
    return out


def count(nU: int, nV: int, u, v, kind: str | int = "degree", rank_of=None,
          per_vertex: bool = True, per_edge: bool = True, nthreads: int | None = None) -> Counts:
    """Exact counts by the paper's ranked wedge method (see module doc)."""
    lib = _load()
    k = RANK_KINDS[kind] if isinstance(kind, str) else int(kind)
    u, pu = _u32(u)
    v, pv_ = _u32(v)
    m_in = u.shape[0]
    n = nU + nV
    W = np.zeros(1, np.uint64)
    g = np.zeros(1, np.uint64)
    m = np.zeros(1, np.uint64)
    pvo = np.zeros(n, np.uint64) if per_vertex else None
    peo = np.zeros(m_in, np.uint64) if per_edge else None
    rk = None
    if rank_of is not None:
        rk, prk = _u32(rank_of)
    rc = lib.orc_count(nU, nV, m_in, pu, pv_, k, prk if rk is not None else None,
                       nthreads or threads(), _u64(W), _u64(g),
                       _u64(pvo) if pvo is not None else None,
                       _u64(peo) if peo is not None else None, _u64(m))
    _check(rc, "orc_count")
    return Counts(nU, int(W[0]), int(g[0]), int(m[0]), pvo, peo)


def wedges(nU: int, nV: int, u, v, kind: str | int = "degree", rank_of=None) -> int:
    """Exact number of wedges GET-WEDGES retrieves under a ranking."""
    lib = _load()
    k = RANK_KINDS[kind] if isinstance(kind, str) else int(kind)
    u, pu = _u32(u)
    v, pv_ = _u32(v)
    W = np.zeros(1, np.uint64)
    prk = None
    if rank_of is not None:
        rk, prk = _u32(rank_of)
    _check(lib.orc_wedges(nU, nV, u.shape[0], pu, pv_, k, prk, _u64(W)), "orc_wedges")
    return int(W[0])


def edge_eq2(nU: int, nV: int, u, v, query) -> np.ndarray:
    """Per-edge butterfly counts of the input edges `query` straight from Eq. 2."""
    lib = _load()
    u, pu = _u32(u)
    v, pv_ = _u32(v)
    q = np.ascontiguousarray(query, dtype=np.uint64)
    out = np.zeros(q.shape[0], np.uint64)
    _check(lib.orc_edge_eq2(nU, nV, u.shape[0], pu, pv_, q.shape[0], _u64(q), 1, _u64(out)),
           "orc_edge_eq2")
    return out


def vertex_eq1(nU: int, nV: int, u, v, query) -> np.ndarray:
    """Per-vertex butterfly counts of the global ids `query` straight from Eq. 1."""
    lib = _load()
    u, pu = _u32(u)
    v, pv_ = _u32(v)
    q = np.ascontiguousarray(query, dtype=np.uint64)
    out = np.zeros(q.shape[0], np.uint64)
    _check(lib.orc_vertex_eq1(nU, nV, u.shape[0], pu, pv_, q.shape[0], _u64(q), _u64(out)), "orc_vertex_eq1")
    return out


def count_range(nU: int, nV: int, u, v, x_lo: int, x_hi: int, kind: str | int = "degree",
                nthreads: int | None = None) -> Counts:
    """Partial counts of the wedges whose first endpoint has rank in [x_lo, x_hi)."""
    lib = _load()
    k = RANK_KINDS[kind] if isinstance(kind, str) else int(kind)
    u, pu = _u32(u)
    v, pv_ = _u32(v)
    m_in = u.shape[0]
    W = np.zeros(1, np.uint64)
    g = np.zeros(1, np.uint64)
    m = np.zeros(1, np.uint64)
    pvo = np.zeros(nU + nV, np.uint64)
    peo = np.zeros(m_in, np.uint64)
    _check(lib.orc_count_range(nU, nV, m_in, pu, pv_, k, None, nthreads or threads(), x_lo, x_hi, _u64(W), _u64(g),
                               _u64(pvo), _u64(peo), _u64(m)), "orc_count_range")
    return Counts(nU, int(W[0]), int(g[0]), int(m[0]), pvo, peo)


def owner_wedges(nU: int, nV: int, u, v, kind: str | int = "degree") -> np.ndarray:
    """Wedges retrieved by each first endpoint, indexed by rank."""
    lib = _load()
    k = RANK_KINDS[kind] if isinstance(kind, str) else int(kind)
    u, pu = _u32(u)
    v, pv_ = _u32(v)
    out = np.zeros(nU + nV, np.uint64)
    _check(lib.orc_owner_wedges(nU, nV, u.shape[0], pu, pv_, k, None, _u64(out)), "orc_owner_wedges")
    return out


"""TEST INFRASTRUCTURE ONLY -- sparsification for approximate counts
(Sec. "Approximate counting"), written independently of the CUDA library.

Edge sparsification keeps each edge with probability p and divides the count
of the kept graph by p^4; colourful sparsification colours every vertex with
one of c = ceil(1/p) colours and keeps the edges whose endpoints share a
colour.  A butterfly then survives when its other three vertices draw the
first one's colour, with probability c^-3 -- the paper's p^3 when 1/p is an
integer -- so the kept count is multiplied by c^3.  Each decision is a uniform draw from SplitMix64's output
function (Steele, Lea & Flood, OOPSLA 2014) applied to the edge or vertex:
h = mix(mix(seed ^ a * 0x9E3779B97F4A7C15) + b), U = (h >> 11) * 2^-53, with
(a, b) = (u, v) for an edge and (global id, 0x5BD1E995) for a colour.
"""
from __future__ import annotations

import math

import numpy as np

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_G = np.uint64(0x9E3779B97F4A7C15)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, a, b):
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = _mix(_mix(np.uint64(seed) ^ (a * _G)) + b)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def keep_mask(nU: int, u, v, kind: str, p: float, seed: int) -> np.ndarray:
    u = np.asarray(u, dtype=np.uint64)
    v = np.asarray(v, dtype=np.uint64)
    if kind == "edge":
        return uniform(seed, u, v) < p
    colors = math.ceil(1.0 / p)
    cu = (uniform(seed, u, 0x5BD1E995) * colors).astype(np.uint64)
    cv = (uniform(seed, np.uint64(nU) + v, 0x5BD1E995) * colors).astype(np.uint64)
    return cu == cv


def sparsify(nU: int, nV: int, u, v, kind: str, p: float, seed: int):
    """Kept pairs in input order, and the estimator's scale factor."""
    k = keep_mask(nU, u, v, kind, p, seed)
    scale = 1.0 / p ** 4 if kind == "edge" else float(math.ceil(1.0 / p)) ** 3
    return np.asarray(u)[k].astype(np.uint32), np.asarray(v)[k].astype(np.uint32), scale

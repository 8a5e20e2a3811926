"""TEST INFRASTRUCTURE ONLY -- butterfly counts straight from their definitions.

For tiny graphs.  No ranking and no wedge aggregation: every quantity is the
definition written out over all vertex pairs.

* A butterfly is two vertices on each side with all four edges between them
  (preliminaries).  For a pair u != u' in U sharing c = |N(u) n N(u')|
  neighbours there are C(c, 2) butterflies containing both, so the global
  count is the sum of C(c, 2) over unordered U pairs -- and equally over
  unordered V pairs.
* Per vertex (Eq. 1): sum over u' != u of C(|N(u) n N(u')|, 2); the paper sums
  over the 2-hop neighbourhood N_2(u), and pairs outside it contribute
  C(0, 2) = 0.
* Per edge (Eq. 2): count(u, v) = sum over u' in N(v) \\ {u} of
  (|N(u) n N(u')| - 1).
* Retrieved wedges under a ranking (Algorithm 2): a wedge with centre y and
  endpoints a, b is retrieved exactly when its lower-ranked endpoint ranks
  below y (the other endpoint then ranks above it by construction).

The pairwise intersection sizes come from one integer matrix product of the
0/1 biadjacency matrix (a library primitive); everything else is loops.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def _adj(nU: int, nV: int, u, v) -> np.ndarray:
    A = np.zeros((nU, nV), dtype=np.float64)
    A[np.asarray(u, np.int64), np.asarray(v, np.int64)] = 1.0  # duplicates collapse
    return A


def _c2(x):
    x = np.asarray(x, dtype=np.int64)
    return x * (x - 1) // 2


def counts(nU: int, nV: int, u, v):
    """(global, per-vertex[nU + nV], per-edge[m_in]) by the definitions."""
    A = _adj(nU, nV, u, v)
    CU = np.rint(A @ A.T).astype(np.int64)   # |N(u) n N(u')|
    CV = np.rint(A.T @ A).astype(np.int64)   # |N(v) n N(v')|
    iu = np.triu_indices(nU, 1)
    iv = np.triu_indices(nV, 1)
    glob_u = int(_c2(CU[iu]).sum())
    glob_v = int(_c2(CV[iv]).sum())
    if glob_u != glob_v:
        raise AssertionError("U-pair and V-pair butterfly totals differ")
    # Eq. 1 per vertex: C(., 2) of the intersection with every other vertex
    # of the same side (the diagonal, the vertex with itself, is excluded).
    PU = _c2(CU)
    np.fill_diagonal(PU, 0)
    PV = _c2(CV)
    np.fill_diagonal(PV, 0)
    pv = np.concatenate([PU.sum(axis=1), PV.sum(axis=1)])
    nbrU = [set(np.nonzero(A[a])[0].tolist()) for a in range(nU)]
    nbrV = [set(np.nonzero(A[:, b])[0].tolist()) for b in range(nV)]
    pe = np.zeros(len(u), dtype=np.int64)
    for k, (a, b) in enumerate(zip(np.asarray(u).tolist(), np.asarray(v).tolist())):
        s = 0
        for a2 in nbrV[b]:
            if a2 != a:
                s += len(nbrU[a] & nbrU[a2]) - 1
        pe[k] = s
    return glob_u, pv, pe


def global_count(nU: int, nV: int, u, v) -> int:
    A = _adj(nU, nV, u, v)
    CU = np.rint(A @ A.T).astype(np.int64)
    return int(_c2(CU[np.triu_indices(nU, 1)]).sum())


def wedges(nU: int, nV: int, u, v, rank_of) -> int:
    """Number of wedges Algorithm 2 retrieves under rank_of[id] (ids U then V)."""
    A = _adj(nU, nV, u, v)
    rank_of = np.asarray(rank_of, dtype=np.int64)
    W = 0
    for b in range(nV):                      # centres in V, endpoints in U
        nb = np.nonzero(A[:, b])[0].tolist()
        ry = rank_of[nU + b]
        for a1, a2 in combinations(nb, 2):
            if min(rank_of[a1], rank_of[a2]) < ry:
                W += 1
    for a in range(nU):                      # centres in U, endpoints in V
        nb = np.nonzero(A[a])[0].tolist()
        ry = rank_of[a]
        for b1, b2 in combinations(nb, 2):
            if min(rank_of[nU + b1], rank_of[nU + b2]) < ry:
                W += 1
    return W


def butterflies_listed(nU: int, nV: int, u, v):
    """Every butterfly as ((u1, u2), (v1, v2)) by exhaustive search (tiny graphs)."""
    A = _adj(nU, nV, u, v) > 0
    out = []
    for a1, a2 in combinations(range(nU), 2):
        common = np.nonzero(A[a1] & A[a2])[0].tolist()
        for b1, b2 in combinations(common, 2):
            out.append(((a1, a2), (b1, b2)))
    return out


def complement_degeneracy_rank(nU: int, nV: int, u, v, approx: bool = False):
    """Peeling rounds written out with sets: every round removes all
    remaining vertices of largest current degree (or largest current
    floor(log2 degree), degree 0 lowest); ties within a round by global id."""
    n = nU + nV
    nbr = [set() for _ in range(n)]
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        nbr[a].add(nU + b)
        nbr[nU + b].add(a)
    remaining = set(range(n))
    rank = np.empty(n, np.int64)
    nxt = 0

    def key(x):
        d = len(nbr[x] & remaining)
        if not approx:
            return d
        return d.bit_length() - 1 if d > 0 else -1

    while remaining:
        best = max(key(x) for x in remaining)
        front = sorted(x for x in remaining if key(x) == best)
        for x in front:
            rank[x] = nxt
            nxt += 1
        remaining -= set(front)
    return rank


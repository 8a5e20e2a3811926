"""Shared input helpers for the tests (inputs only, no counting)."""
import numpy as np

import synth


def fig2_graph(fx):
    """(nU, nV, u, v, name_to_gid) of the paper's Fig. 1 graph from its fixture."""
    U, V = fx["vertices"]["U"], fx["vertices"]["V"]
    gid = {name: i for i, name in enumerate(U)}
    gid.update({name: len(U) + j for j, name in enumerate(V)})
    u = np.array([U.index(a) for a, b in fx["edges"]], np.uint32)
    v = np.array([V.index(b) for a, b in fx["edges"]], np.uint32)
    return len(U), len(V), u, v, gid


def fig2_rank(fx, gid):
    """rank_of[gid] for the Step 1 ranking of Fig. 2."""
    r = np.empty(len(gid), np.uint32)
    for pos, name in enumerate(fx["ranking_step1"]):
        r[gid[name]] = pos
    return r


def tiny_graphs(count=60, seed=0x51A7):
    """Seeded tiny graphs: Erdos-Renyi and Chung-Lu, varied shapes and densities."""
    out = []
    for i in range(count):
        s = seed * 1000 + i
        nU = 2 + int(synth.uniform(s, 7, 0) * 30)
        nV = 2 + int(synth.uniform(s, 7, 1) * 30)
        dens = 0.05 + 0.45 * synth.uniform(s, 7, 2)
        m = max(1, min(int(dens * nU * nV), nU * nV // 2))
        if i % 2 == 0:
            g = synth.er_graph(s, nU, nV, m)
        else:
            g = synth.chung_lu_graph(s, nU, nV, m, 1.8 + synth.uniform(s, 7, 3), 2.2,
                                     cap_u=max(1.0, nV / 2), cap_v=max(1.0, nU / 2))
        out.append(g)
    return out


def random_rank(seed, n):
    """A seeded random permutation used as an arbitrary ranking."""
    keys = np.array([synth.draw(seed, 9, i) for i in range(n)], dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    r = np.empty(n, np.uint32)
    r[order] = np.arange(n, dtype=np.uint32)
    return r

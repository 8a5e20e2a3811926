"""Writes tests/golden/cl3_oracle.json: the oracle's complete counts on the
Chung-Lu |U|=20M, |V|=60M, m=3e8 workload, stored as digests.

The full per-vertex (80M) and per-edge (3e8) arrays are too large to keep in
the repository, so the file holds the wedge count W under degree order, the
global count, SHA-256 digests of the per-vertex array (U ids then V ids) and of
the per-edge array (input order), both as little-endian uint64, and a few
sampled entries for readable failure messages.  Every value comes from
`oracle.count`; the input from `synth.workload(3)`.

Run once on a machine with ~40 GB of RAM (about an hour on 8 cores):
    python tests/golden/make_cl3_oracle.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def main():
    t0 = time.time()
    g = synth.workload(3)
    t1 = time.time()
    ref = oracle.count(g.nU, g.nV, g.u, g.v, kind="degree")
    t2 = time.time()
    pick_v = [int(synth.draw(0xC3, 12, i) % (g.nU + g.nV)) for i in range(16)]
    pick_e = [int(synth.draw(0xE3, 12, i) % g.m) for i in range(16)]
    out = {
        "workload": g.name, "nU": g.nU, "nV": g.nV, "m": int(g.m),
        "ranking": "degree", "W": ref.W, "global": ref.global_count,
        "per_vertex_sha256": digest(ref.per_vertex), "per_edge_sha256": digest(ref.per_edge),
        "per_vertex_sum": int(ref.per_vertex.sum(dtype=np.uint64)),
        "per_edge_sum": int(ref.per_edge.sum(dtype=np.uint64)),
        "samples_vertex": {str(i): int(ref.per_vertex[i]) for i in pick_v},
        "samples_edge": {str(i): int(ref.per_edge[i]) for i in pick_e},
        "oracle_threads": oracle.threads(),
        "seconds": {"generate": round(t1 - t0, 1), "oracle": round(t2 - t1, 1)},
    }
    with open(os.path.join(ROOT, "tests", "golden", "cl3_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()

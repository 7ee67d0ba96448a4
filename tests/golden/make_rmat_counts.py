"""Writes rmat_counts.json: exact triangle and 4-cycle counts of seeded
R-MAT graphs (a, b, c = 0.57, 0.19, 0.19; 16 edges per vertex; seed 3),
computed by the oracle's Generic Join alone.  Run from the repository root:

    python tests/golden/make_rmat_counts.py

Scale 14 counts both queries; scales 16 and 18 count triangles only (the
oracle's 4-cycle count at scale 14 already takes minutes)."""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2301_10841_gb300 import datagen as G  # noqa: E402


def main():
    oracle.build()
    out = {"_about": "Exact counts on seeded R-MAT graphs: Q_tri(x,y,z) :- E(x,y),E(y,z),E(z,x) "
                     "and Q_4(w,x,y,z) :- E(w,x),E(x,y),E(y,z),E(z,w) (bag semantics, every "
                     "directed cycle counted once per rotation), written by this script from "
                     "the oracle's Generic Join (Section 2.3).  Graph: datagen.rmat(scale, "
                     "16 << scale, seed=3).",
           "graphs": []}
    for scale, four in ((14, True), (16, False), (18, False)):
        e = G.rmat(scale, 16 << scale, seed=3)
        rec = {"scale": scale, "n_edges": 16 << scale, "seed": 3}
        t0 = time.time()
        rec["triangles"] = int(oracle.generic_join(G.triangle_query(e))[0])
        if four:
            rec["four_cycles"] = int(oracle.generic_join(G.four_cycle_query(e))[0])
        rec["oracle_seconds"] = round(time.time() - t0, 1)
        out["graphs"].append(rec)
        print(rec, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat_counts.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

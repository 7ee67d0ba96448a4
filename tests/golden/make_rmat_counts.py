"""Writes rmat_counts.json: exact triangle and 4-cycle counts of seeded
R-MAT graphs (a, b, c = 0.57, 0.19, 0.19; 16 edges per vertex; seed 3),
computed by the oracle's Generic Join alone.  Run from the repository root:

    python tests/golden/make_rmat_counts.py

Scale 14 counts both queries; scales 16 and 18 count triangles only (the
oracle's 4-cycle enumeration at scale 14 already takes minutes).  The
4-cycles are also counted by the 2-path form (oracle.closed.
four_cycles_two_paths, sparse integer products) at every scale it reaches
in memory; `--two-paths-only` adds those counts to the existing file
without recounting the rest, and `--full-size` adds the 4-cycle count of
the full-size graph (scale 20) the same way."""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import closed  # noqa: E402
from paper_2301_10841_gb300 import datagen as G  # noqa: E402


TWO_PATH_SCALES = (14, 16, 18)
ABOUT = ("Exact counts on seeded R-MAT graphs: Q_tri(x,y,z) :- E(x,y),E(y,z),E(z,x) "
         "and Q_4(w,x,y,z) :- E(w,x),E(x,y),E(y,z),E(z,w) (bag semantics, every "
         "directed cycle counted once per rotation), written by this script from "
         "the oracle's Generic Join (Section 2.3); four_cycles_two_paths from the "
         "2-path form sum_{w,y} P2[w,y] P2[y,w] (oracle.closed).  Graph: "
         "datagen.rmat(scale, 16 << scale, seed=3).")


def two_paths(rec):
    e = G.rmat(rec["scale"], rec["n_edges"], seed=rec["seed"])
    t0 = time.time()
    rec["four_cycles_two_paths"] = closed.four_cycles_two_paths(e["cols"][0], e["cols"][1],
                                                                1 << rec["scale"])
    rec["two_paths_seconds"] = round(time.time() - t0, 1)
    print(rec, flush=True)


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat_counts.json")
    if "--two-paths-only" in sys.argv or "--full-size" in sys.argv:
        with open(path) as f:
            out = json.load(f)
        out["_about"] = ABOUT
        if "--full-size" in sys.argv:
            # The full-size graph (2^20 vertices, 2^24 edges): 4-cycles by
            # the 2-path form only (about half an hour on one host core).
            rec = {"scale": 20, "n_edges": 16 << 20, "seed": 3}
            two_paths(rec)
            out["full_size"] = rec
        else:
            for rec in out["graphs"]:
                if rec["scale"] in TWO_PATH_SCALES:
                    two_paths(rec)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        return
    oracle.build()
    out = {"_about": ABOUT, "graphs": []}
    for scale, four in ((14, True), (16, False), (18, False)):
        e = G.rmat(scale, 16 << scale, seed=3)
        rec = {"scale": scale, "n_edges": 16 << scale, "seed": 3}
        t0 = time.time()
        rec["triangles"] = int(oracle.generic_join(G.triangle_query(e))[0])
        if four:
            rec["four_cycles"] = int(oracle.generic_join(G.four_cycle_query(e))[0])
        rec["oracle_seconds"] = round(time.time() - t0, 1)
        if scale in TWO_PATH_SCALES:
            two_paths(rec)
        out["graphs"].append(rec)
        print(rec, flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

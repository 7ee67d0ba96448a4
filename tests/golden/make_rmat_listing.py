"""Writes rmat_listing.json: the oracle's listing of the triangles of the
full-size R-MAT graph (scale 20, 2^24 edges, seed 3) whose x lies below a
small cutoff, as its count, a SHA-256 of the sorted (x, y, z) int32 rows and
the first and last rows.  Computed by the oracle's hash join alone, with the
selection x < cutoff pushed into E1(x, y) and E3(z, x).  Run from the
repository root:

    python tests/golden/make_rmat_listing.py
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
from paper_2301_10841_gb300 import datagen as G  # noqa: E402

CUTOFFS = (64, 512)


def main():
    oracle.build()
    e = G.rmat(20, 16 << 20, seed=3)
    out = {"_about": "Triangles Q(x,y,z) :- E(x,y),E(y,z),E(z,x) of datagen.rmat(20, 16 << 20, "
                     "seed=3) with x < cutoff, listed by the oracle's hash join (Section 2.2) and "
                     "sorted lexicographically; sha256 over the rows as little-endian int32.",
           "listings": []}
    for cutoff in CUTOFFS:
        atoms = []
        for a in G.triangle_query(e):
            b = dict(a)
            b["preds"] = [(a["vars"].index(0), "<", cutoff)] if 0 in a["vars"] else []
            atoms.append(b)
        t0 = time.time()
        cnt, _, rows = oracle.binary_join(atoms, head=[0, 1, 2], materialize=True)
        rows = np.ascontiguousarray(rows, dtype="<i4")
        rec = {"cutoff": cutoff, "count": int(cnt),
               "sha256": hashlib.sha256(rows.tobytes()).hexdigest(),
               "first": rows[:5].tolist(), "last": rows[-5:].tolist(),
               "oracle_seconds": round(time.time() - t0, 1)}
        out["listings"].append(rec)
        print(rec["cutoff"], rec["count"], rec["oracle_seconds"], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat_listing.json"),
              "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

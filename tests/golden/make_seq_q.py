"""Writes tests/golden/rmat22_seq_q.json: the modularity that the oracle's
sequential Louvain (one vertex at a time in id order, every move updating the
community totals at once, Section 3.3's loop; aggregation between passes)
reaches on the seeded R-MAT scale-22 graph (edge factor 16,
(0.57, 0.19, 0.19, 0.05), weights in [1, 16], seed 1) with the k-slot
sketch (Algorithm 1, one stream per row in stored order).

Calls only oracle/ (and the seeded input generator); nothing here comes from
the CUDA path.  Run from the repository root:
    python tests/golden/make_seq_q.py [k ...]      (default: 8)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2411_02268_gb300 import gen  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat22_seq_q.json")


def main(ks):
    g = gen.rmat22(1)
    try:
        with open(OUT) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data["_source"] = ("oracle.louvain_seq (sequential Gauss-Seidel Louvain, default tolerances: 0.01 "
                       "divided by 10 per pass, 20 sweeps per pass, 10 passes, stop when |V'| > 0.8 |V|) "
                       "on R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), w in [1,16], seed 1; "
                       "written by tests/golden/make_seq_q.py")
    data["graph"] = {"n": g.n, "nnz": g.nnz, "checksum": gen.checksum(g)}
    for k in ks:
        t = time.time()
        lab = oracle.louvain_seq(g, k=k)
        fr = oracle.modularity_fraction(g, lab)
        data[f"k{k}"] = {"q": float(fr), "q_num": str(fr.numerator), "q_den": str(fr.denominator),
                         "communities": int(lab.max()) + 1, "seconds": round(time.time() - t, 1)}
        print(k, data[f"k{k}"], flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)


if __name__ == "__main__":
    main([int(x) for x in sys.argv[1:]] or [8])

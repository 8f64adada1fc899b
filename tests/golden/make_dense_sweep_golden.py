"""Write the FP64 oracle's outcome on every path of the dense total-degree
sweep (quadratics n = 8, 10, 12; cubics n = 6, 8; 16 systems per size) to
dense_sweep_oracle.json beside this script.

Calls only the oracle (and the seeded input generator).  Per system it
stores the status counts per class, the number of distinct finite roots
(relative infinity distance > 1e-6), and the path ids and statuses of every
path the oracle does not end at a finite root.  Run:

    python tests/golden/make_dense_sweep_golden.py [--threads T]

Takes about ten minutes on eight cores.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from hcmatch import distinct  # noqa: E402
from paper_2112_03444_gb300 import inputs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "dense_sweep_oracle.json"))
    args = ap.parse_args()
    classes = []
    t0 = time.time()
    for w in inputs.dense_sweep(0):
        n, d = w["n"], w["d"]
        systems = []
        for k, seed in enumerate(w["seeds"]):
            pr = oracle.OracleProblem(w["base"], gamma=w["gamma"], coef=w["coefs"][k])
            r = pr.track(threads=args.threads)
            st = r["status"]
            fin = (st & 0x7F) == oracle.FINITE
            bad = np.nonzero(~fin)[0]
            systems.append(dict(seed=int(seed), counts=oracle.status_counts(st),
                                distinct_finite=int(distinct(r["x"][fin], 1e-6)),
                                max_be=float(np.max(r["be"][fin])) if fin.any() else None,
                                not_finite=[[int(i), int(st[i])] for i in bad]))
            print(f"n={n} d={d} seed={seed}: {systems[-1]['counts']} "
                  f"({time.time() - t0:.0f} s)", flush=True)
        classes.append(dict(n=n, d=d, paths=d ** n, gamma=[w["gamma"].real, w["gamma"].imag],
                            systems=systems))
    doc = dict(what="FP64 oracle on every path of the dense total-degree sweep (default "
                    "settings, RK4 + <= 3 Newton, dt in [1e-6, 0.05])",
               generator="tests/golden/make_dense_sweep_golden.py", classes=classes)
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()

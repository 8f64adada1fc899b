"""Writes the start-solution sets of the parameter-homotopy workloads.

Runs the oracle's monodromy solver (oracle/monodromy.py, FP64 C++ tracking)
once per problem family and stores the result as an input file:
  paper_2112_03444_gb300/startsets/<family>.npz
with arrays start [S, n] complex128, p0 [P] complex128, and the loop log.
Usage:  python -m oracle.make_start_sets [triangulation4] [trifocal_f] [triangulation2]
                                         [p3p] [pose5_depth]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import monodromy  # noqa: E402
from paper_2112_03444_gb300 import inputs  # noqa: E402

OUT = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")
FAMILIES = {"triangulation4": lambda: inputs.triangulation_family(4),
            "trifocal_f": inputs.trifocal_family,
            "triangulation2": lambda: inputs.triangulation_family(2),
            "p3p": inputs.p3p_family,
            "pose5_depth": inputs.pose5_depth_family}


def make(name, seed=0, stall_loops=10, threads=0):
    fam = FAMILIES[name]()
    t0 = time.time()
    S, p0, log = monodromy.solve(fam, seed=seed, stall_loops=stall_loops, threads=threads,
                                 verbose=True)
    res = max(float(np.max(np.abs(monodromy.residual(fam.system, x, p0)))) for x in S)
    os.makedirs(OUT, exist_ok=True)
    path = os.path.join(OUT, f"{name}.npz")
    np.savez_compressed(path, start=S, p0=p0, seed=seed, stall_loops=stall_loops,
                        log=json.dumps(log), max_residual=res)
    print(f"{name}: {len(S)} solutions, max residual {res:.2e}, {time.time() - t0:.0f} s -> {path}")
    return path


if __name__ == "__main__":
    names = sys.argv[1:] or list(FAMILIES)
    for nm in names:
        make(nm)

"""Write the FP64 oracle's outcome on every one of the 5344 trifocal start
paths for two seeded noisy scenes to trifocal_oracle.npz beside this script.

Calls only the oracle (and the seeded input generators).  Per scene and
path: the status code, the random linear projection l(x) = sum_i c_i x_i of
the endpoint (c: unit-modulus complex numbers drawn from seed 2112) and its
infinity norm -- enough to match every finite GPU endpoint to an oracle
endpoint within the 1e-8 relative bound, since |l(a) - l(b)| <=
sum_i |c_i| * max_i |a_i - b_i|.  Run:

    python tests/golden/make_trifocal_golden.py [--threads T]

Takes a few minutes on eight cores.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2112_03444_gb300 import inputs  # noqa: E402

SCENES = (53, 54)


def projection(n):
    rng = np.random.default_rng(2112)
    return np.exp(2j * np.pi * rng.uniform(size=n))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "trifocal_oracle.npz"))
    args = ap.parse_args()
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(ROOT, "paper_2112_03444_gb300", "startsets", "trifocal_f.npz"))
    c = projection(fam.system.n)
    out = dict(scenes=np.array(SCENES), proj_coef=c)
    for k, seed in enumerate(SCENES):
        p1 = inputs.trifocal_scene(seed)[0]
        t0 = time.time()
        r = oracle.OracleProblem(fam.system, kind=oracle.KIND_PARAMETER, p0=z["p0"],
                                 p1=p1).track(start=z["start"], threads=args.threads)
        out[f"status{k}"] = r["status"]
        out[f"proj{k}"] = r["x"] @ c
        out[f"xnorm{k}"] = np.max(np.abs(r["x"]), axis=1)
        print(f"scene {seed}: {oracle.status_counts(r['status'])} ({time.time() - t0:.0f} s)",
              flush=True)
    np.savez_compressed(args.out, **out)
    print("wrote", args.out)


if __name__ == "__main__":
    main()

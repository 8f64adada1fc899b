"""Monodromy solver for start solutions of a parameter homotopy (oracle side).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): it produces the start
solution sets that the parameter-homotopy workloads consume, by tracking
with the FP64 C++ oracle; nothing here runs on the GPU path.

Paper, Sec. 7: the start systems of the vision problems come from the
monodromy module of Macaulay2 at a generic complex parameter point.  The
method, written here from its description:
  1. seed pair: a random complex x0 and parameters p0 with F(x0; p0) = 0,
     obtained by solving for the parameters in which F is affine (for the
     triangulation family the essential-matrix entries, for the trifocal
     family the image points of views 2 and 3);
  2. loops p0 -> pa -> pb -> p0 through random complex parameter points
     (parameter homotopies; the random complex detour plays the role of the
     gamma trick); every known solution is tracked around the loop, and the
     endpoints not yet known are added;
  3. stop after `stall_loops` consecutive loops that add nothing.
The solution count is recorded, not assumed.
"""
from __future__ import annotations

import time

import numpy as np

from . import FINITE, KIND_PARAMETER, OracleProblem


def _complex_normal(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def residual(system, x, p):
    pr = OracleProblem(system, kind=KIND_PARAMETER, p0=p, p1=p)
    return pr.eval(np.asarray(x, np.complex128), 1.0)[0]


def seed_pair(family, rng):
    """(x0, p0) with F(x0; p0) = 0 for a random complex x0 (step 1)."""
    sys_ = family.system
    n, P = sys_.n, sys_.n_params
    x0 = _complex_normal(rng, n)
    for grp in family.unit_groups:
        q = x0[grp]
        x0[grp] = q / np.sqrt(np.sum(q * q))
    p = _complex_normal(rng, P)
    lin = list(family.linear_params)
    p[lin] = 0.0
    if family.complete_seed is not None:
        # equations in no linear parameter: the family fixes x0 to satisfy them
        x0 = family.complete_seed(x0, p)
    r = residual(sys_, x0, p)
    A = np.zeros((n, len(lin)), np.complex128)
    for c, l in enumerate(lin):
        q = p.copy()
        q[l] = 1.0
        A[:, c] = residual(sys_, x0, q) - r
    rows = np.where(np.max(np.abs(A), axis=1) > 0)[0]
    Ar, br = A[rows], -r[rows]
    # minimum-norm solution plus a random null-space component
    y = Ar.conj().T @ np.linalg.solve(Ar @ Ar.conj().T, br)
    z = _complex_normal(rng, len(lin))
    z = z - Ar.conj().T @ np.linalg.solve(Ar @ Ar.conj().T, Ar @ z)
    p[lin] = y + z
    return x0, p


def _new_points(X, known, tol):
    out = []
    for x in X:
        sc = max(1.0, float(np.max(np.abs(x))))
        if known is not None and len(known):
            d = np.max(np.abs(known - x), axis=1)
            if np.min(d) <= tol * sc:
                continue
        if out:
            d = np.max(np.abs(np.array(out) - x), axis=1)
            if np.min(d) <= tol * sc:
                continue
        out.append(x)
    return out


def solve(family, seed=0, stall_loops=10, max_loops=400, threads=0, settings=None,
          tol=1e-6, verbose=False):
    """Monodromy solve: returns (start solutions [S, n], p0, log)."""
    rng = np.random.default_rng([seed, 0x30D0])
    sys_ = family.system
    x0, p0 = seed_pair(family, rng)
    S = np.array([x0])
    stall, loops, tracked = 0, 0, 0
    log = []
    t0 = time.time()
    while stall < stall_loops and loops < max_loops:
        pa = _complex_normal(rng, sys_.n_params)
        pb = _complex_normal(rng, sys_.n_params)
        X = S.copy()
        for (pf, pt) in ((p0, pa), (pa, pb), (pb, p0)):
            if len(X) == 0:
                break
            r = OracleProblem(sys_, kind=KIND_PARAMETER, p0=pf, p1=pt).track(
                start=X, settings=settings, threads=threads)
            tracked += len(X)
            X = r["x"][(r["status"] & 0x7F) == FINITE]
        new = _new_points(X, S, tol)
        loops += 1
        if new:
            S = np.concatenate([S, np.array(new)])
            stall = 0
        else:
            stall += 1
        log.append(dict(loop=loops, known=len(S), new=len(new), tracked=tracked,
                        seconds=time.time() - t0))
        if verbose:
            print(log[-1], flush=True)
    return S, p0, log

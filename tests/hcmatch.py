"""Set comparison of endpoint lists (test helper).

A homotopy returns a *set* of roots: path order may permute when paths jump,
so parity is a bijective matching by relative infinity-norm distance plus
exact counts per status class.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def rel_dist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """max_i |a_i - b_i| / max(1, ||b||_inf), row-wise."""
    a = np.atleast_2d(a)
    b = np.atleast_2d(b)
    return np.max(np.abs(a - b), axis=1) / np.maximum(1.0, np.max(np.abs(b), axis=1))


def _embed(x):
    x = np.atleast_2d(np.asarray(x, np.complex128))
    return np.concatenate([x.real, x.imag], axis=1)


def match(a, b, tol):
    """Match rows of a to rows of b.

    Returns (perm, dist): perm[i] = index in b of the nearest row to a[i]
    (by infinity norm on the real embedding), dist[i] = rel_dist there.
    """
    a = np.atleast_2d(np.asarray(a, np.complex128))
    b = np.atleast_2d(np.asarray(b, np.complex128))
    if len(a) == 0 or len(b) == 0:
        return np.zeros(len(a), np.int64), np.full(len(a), np.inf)
    tree = cKDTree(_embed(b))
    _, idx = tree.query(_embed(a), k=1, p=np.inf)
    d = rel_dist(a, b[idx])
    return idx, d


def same_set(a, b, tol):
    """True iff a and b have equal size and match bijectively within tol."""
    a = np.atleast_2d(np.asarray(a, np.complex128))
    b = np.atleast_2d(np.asarray(b, np.complex128))
    if a.shape != b.shape:
        return False, f"sizes differ: {a.shape} vs {b.shape}"
    if len(a) == 0:
        return True, "empty"
    idx, d = match(a, b, tol)
    if np.max(d) > tol:
        return False, f"max rel dist {np.max(d):.3e} > {tol:g} at row {int(np.argmax(d))}"
    if len(np.unique(idx)) != len(idx):
        return False, "matching is not bijective (duplicate targets)"
    return True, f"max rel dist {np.max(d):.3e}"


def distinct(x, tol=1e-6):
    """Number of distinct rows (relative infinity distance > tol)."""
    x = np.atleast_2d(np.asarray(x, np.complex128))
    if len(x) == 0:
        return 0
    emb = _embed(x)
    scale = np.maximum(1.0, np.max(np.abs(x), axis=1))
    tree = cKDTree(emb)
    reps = []
    taken = np.zeros(len(x), bool)
    for i in range(len(x)):
        if taken[i]:
            continue
        nb = tree.query_ball_point(emb[i], r=tol * scale[i], p=np.inf)
        taken[nb] = True
        reps.append(i)
    return len(reps)

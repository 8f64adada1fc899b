"""The bench's accounting on CPU: the algorithmic flop model behind the
roofline against closed forms, and the oracle-matched path count behind the
headline value on hand-made status tables (matched, oracle-only, GPU-only,
a root reported twice)."""
import os
import sys
from math import comb

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _distinct_variable_sum(n, d):
    """sum over the monomials of degree <= d of their number of distinct
    variables, by counting monomial shapes: degree 1: x_i; degree 2: x_i^2
    (1 variable), x_i x_j (2); degree 3: x_i^3 (1), x_i^2 x_j (2), x_i x_j x_k (3)."""
    s = 0
    if d >= 1:
        s += n
    if d >= 2:
        s += n * 1 + comb(n, 2) * 2
    if d >= 3:
        s += n * 1 + n * (n - 1) * 2 + comb(n, 3) * 3
    return s


@pytest.mark.parametrize("n,d", [(1, 2), (6, 2), (8, 2), (10, 2), (12, 2),
                                 (2, 3), (6, 3), (8, 3)])
def test_flop_model_matches_closed_forms(n, d):
    f = bench.dense_flops_per_unit(n, d)
    assert f["E_H"] == n * comb(n + d, d)
    assert f["E_Ht"] == f["E_H"]
    assert f["E_Hx"] == n * _distinct_variable_sum(n, d)
    if d == 2:  # every monomial of degree <= 1 is a variable or the constant
        assert f["E_Hx"] == n * n * (n + 1)
    # augmented LU of an n x (n+1) matrix, sum_{j<n} j (j + 1) = (n-1) n (n+1) / 3,
    # plus the back substitution n (n+1) / 2
    assert f["S"] == (n - 1) * n * (n + 1) // 3 + n * (n + 1) // 2


def test_flop_model_cubic_n8_values():
    # the dominant class of the sweep: 2880 cFMA for the Jacobian, 1320 for
    # H (165 monomials x 8 equations), 204 for the solve
    assert bench.dense_flops_per_unit(8, 3) == dict(E_H=1320, E_Ht=1320, E_Hx=2880, S=204)
    # one RK4 step (4 stages of Hx, Ht and a solve) and one Newton iteration
    # (H, Hx and a solve), 8 flops per complex FMA
    assert bench.flops(8, 3, 1, 0) == 8.0 * 4 * (2880 + 1320 + 204)
    assert bench.flops(8, 3, 0, 1) == 8.0 * (1320 + 2880 + 204)


def _workload():
    return [dict(n=2, d=2, seeds=[11, 12]), dict(n=1, d=3, seeds=[21])]


def _golden(not_finite):
    return dict(classes=[
        dict(systems=[dict(seed=11, not_finite=not_finite.get((0, 0), [])),
                      dict(seed=12, not_finite=not_finite.get((0, 1), []))]),
        dict(systems=[dict(seed=21, not_finite=not_finite.get((1, 0), []))]),
    ])


def _roots(k, n, offset):
    """k well-separated points of C^n"""
    return np.array([[complex(offset + 3.0 * i, 1.0 + j) for j in range(n)]
                     for i in range(k)])


def test_match_counts_paths_finite_on_both_sides():
    wl = _workload()
    st = [np.array([[1, 1, 1, 0x81], [1, 2, 1, 1]], np.uint8),  # 0x81: finite and real
          np.array([[1, 3, 1]], np.uint8)]
    xs = [np.stack([_roots(4, 2, 0.0), _roots(4, 2, 50.0)]), _roots(3, 1, 0.0)[None]]
    # the oracle fails path 2 of system (0, 0) and path 2 of system (1, 0)
    golden = _golden({(0, 0): [[2, 3]], (1, 0): [[2, 3]]})
    m = bench.match_sweep(wl, st, xs, golden)
    assert m["total"] == 11
    assert m["gpu_finite"] == 4 + 3 + 2
    assert m["oracle_finite"] == 11 - 2
    # (0,0): paths 0, 1, 3 on both sides; (0,1): 0, 2, 3 (the GPU lost path 1,
    # the oracle did not); (1,0): path 0 (the GPU failed path 1, the oracle
    # path 2)
    assert m["matched"] == 3 + 3 + 1
    assert sorted(m["oracle_only"]) == [[1, 3, 0, 1, 3], [2, 2, 1, 1, 2]]
    assert m["gpu_only"] == 2  # path 2 of (0,0) and of (1,0): finite on the GPU only
    assert m["systems_with_duplicate_roots"] == 0


def test_match_counts_nothing_in_a_system_with_a_root_reported_twice():
    wl = _workload()
    st = [np.ones((2, 4), np.uint8), np.ones((1, 3), np.uint8)]
    x00 = _roots(4, 2, 0.0)
    x00[3] = x00[1] * (1 + 1e-9)  # a path that jumped onto another path's root
    xs = [np.stack([x00, _roots(4, 2, 50.0)]), _roots(3, 1, 0.0)[None]]
    m = bench.match_sweep(wl, st, xs, _golden({}))
    assert m["systems_with_duplicate_roots"] == 1
    assert m["matched"] == 4 + 3  # system (0, 0) counts for nothing
    assert m["oracle_finite"] == 11


def test_match_refuses_a_golden_of_other_seeds():
    wl = _workload()
    wl[0]["seeds"] = [11, 13]
    st = [np.ones((2, 4), np.uint8), np.ones((1, 3), np.uint8)]
    xs = [np.stack([_roots(4, 2, 0.0), _roots(4, 2, 50.0)]), _roots(3, 1, 0.0)[None]]
    with pytest.raises(AssertionError):
        bench.match_sweep(wl, st, xs, _golden({}))


def test_stored_golden_describes_the_benchmarked_sweep():
    golden = bench.load_golden()
    assert golden is not None
    wl = bench.workload(0)
    assert len(golden["classes"]) == len(wl)
    for gc, w in zip(golden["classes"], wl):
        assert [s["seed"] for s in gc["systems"]] == list(w["seeds"])
        for s in gc["systems"]:
            for p, code in s["not_finite"]:
                assert 0 <= p < w["d"] ** w["n"] and (code & 0x7F) != 1

"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against the mathematics (closed forms, library
routines, brute force, invariants), never against a retyping of its own
formula, so that a dropped term, wrong sign, wrong index or transposed
operand anywhere in it fails at least one test.
"""
import cmath
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import OracleProblem, KIND_PARAMETER, KIND_TOTAL_DEGREE
from paper_2112_03444_gb300 import inputs
from hcmatch import same_set, distinct

TOL = 1e-10


def poly_system(n, polys):
    return inputs.system_from_polys(n, polys)


# ---------------------------------------------------------------- start system
@pytest.mark.parametrize("n,d", [(1, 5), (3, 3), (4, 2), (2, 7)])
def test_start_points_are_all_distinct_roots_of_unity(n, d):
    """Closed form: x_i^d = 1 and the d^n start points are pairwise distinct."""
    pr = OracleProblem(inputs.dense_system(n, d, 1))
    P = pr.total_degree_paths()
    assert P == d ** n
    X = np.array([pr.start_point(k) for k in range(P)])
    assert np.max(np.abs(X ** d - 1.0)) < 1e-13
    assert distinct(X, 1e-9) == P
    # variable 1 is the least significant digit of the path index
    assert abs(X[1, 0] - cmath.exp(2j * math.pi / d)) < 1e-15
    if n > 1:
        assert abs(X[1, 1] - 1.0) < 1e-15
        assert abs(X[d, 1] - cmath.exp(2j * math.pi / d)) < 1e-15


def test_start_points_mixed_degrees():
    """Mixed radix for unequal degrees (2, 3): 6 distinct points, x_i^{d_i} = 1."""
    sys_ = poly_system(2, [{(2, 0): 1.0, (0, 0): -3.0}, {(0, 3): 1.0, (1, 0): 2.0}])
    pr = OracleProblem(sys_)
    assert pr.total_degree_paths() == 6
    X = np.array([pr.start_point(k) for k in range(6)])
    assert np.max(np.abs(X[:, 0] ** 2 - 1)) < 1e-14
    assert np.max(np.abs(X[:, 1] ** 3 - 1)) < 1e-14
    assert distinct(X) == 6


# ---------------------------------------------------------------- linear solve
def test_lu_2x2_cramer():
    A = np.array([[1 + 2j, 3 - 1j], [0.5j, -2 + 0.25j]])
    b = np.array([1 - 1j, 2 + 3j])
    det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
    want = np.array([(b[0] * A[1, 1] - A[0, 1] * b[1]) / det,
                     (A[0, 0] * b[1] - b[0] * A[1, 0]) / det])
    x, ok = oracle.solve(A, b)
    assert ok
    assert np.max(np.abs(x - want)) < 1e-14


def test_lu_3x3_cramer_needs_pivoting():
    # zero leading entry: fails without a row interchange
    A = np.array([[0, 2 + 1j, 1], [1j, 1, -1], [3, 0.5, 2 - 1j]], complex)
    b = np.array([1, 2j, -1 + 1j])
    det = np.linalg.det(A)
    want = []
    for j in range(3):
        Aj = A.copy()
        Aj[:, j] = b
        want.append(np.linalg.det(Aj) / det)
    x, ok = oracle.solve(A, b)
    assert ok
    assert np.max(np.abs(x - np.array(want))) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 5, 12, 18, 32])
def test_lu_matches_numpy(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, ok = oracle.solve(A, b)
    assert ok
    want = np.linalg.solve(A, b)
    assert np.max(np.abs(x - want)) / np.max(np.abs(want)) < 1e-11


def test_lu_reports_exactly_singular():
    A = np.array([[1, 2], [2, 4]], complex)
    _, ok = oracle.solve(A, np.array([1, 1], complex))
    assert not ok


# ---------------------------------------------------------------- evaluation
def test_eval_hand_polynomials_and_homotopy_ends():
    """F written out by hand; H(.,1) = F, H(.,0) = gamma*G, Ht = F - gamma*G."""
    # F1 = 3 x1^2 x2 - (2+i) x2 + 5,  F2 = x1 x2 - 4 x1 + 1j
    sys_ = poly_system(2, [{(2, 1): 3.0, (0, 1): -(2 + 1j), (0, 0): 5.0},
                           {(1, 1): 1.0, (1, 0): -4.0, (0, 0): 1j}])
    g = cmath.exp(0.7j)
    pr = OracleProblem(sys_, gamma=g)
    x1, x2 = 0.3 - 0.8j, -1.1 + 0.4j
    F = np.array([3 * x1 ** 2 * x2 - (2 + 1j) * x2 + 5, x1 * x2 - 4 * x1 + 1j])
    J = np.array([[6 * x1 * x2, 3 * x1 ** 2 - (2 + 1j)], [x2 - 4, x1]])
    G = np.array([x1 ** 3 - 1, x2 ** 2 - 1])      # degrees 3 and 2
    Gx = np.diag([3 * x1 ** 2, 2 * x2])
    for t in (0.0, 0.37, 1.0):
        H, Hx, Ht = pr.eval(np.array([x1, x2]), t)
        assert np.max(np.abs(H - ((1 - t) * g * G + t * F))) < 1e-13
        assert np.max(np.abs(Hx - ((1 - t) * g * Gx + t * J))) < 1e-13
        assert np.max(np.abs(Ht - (F - g * G))) < 1e-13


@pytest.mark.parametrize("kind", [KIND_TOTAL_DEGREE, KIND_PARAMETER])
def test_eval_derivatives_by_finite_differences(kind):
    """Hx and Ht against central differences of H (holomorphic in x)."""
    rng = np.random.default_rng(3)
    if kind == KIND_TOTAL_DEGREE:
        sys_ = inputs.dense_system(3, 3, 7)
        pr = OracleProblem(sys_, gamma=inputs.unit_gamma(7))
    else:
        # coefficients polynomial in 3 parameters
        sys_ = inputs.dense_system(3, 2, 8)
        T = sys_.n_terms
        sys_.term_param = rng.integers(-1, 3, size=(T, 3)).astype(np.int32)
        sys_.n_params = 3
        pr = OracleProblem(sys_, kind=KIND_PARAMETER, p0=inputs.random_complex(3, 1),
                           p1=inputs.random_complex(3, 2))
    x = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    t = 0.41
    H, Hx, Ht = pr.eval(x, t)
    h = 1e-6
    for j in range(3):
        for hh in (h, 1j * h):
            e = np.zeros(3, complex)
            e[j] = hh
            fd = (pr.eval(x + e, t)[0] - pr.eval(x - e, t)[0]) / (2 * hh)
            assert np.max(np.abs(fd - Hx[:, j])) < 1e-7 * (1 + np.max(np.abs(Hx)))
    fdt = (pr.eval(x, t + h)[0] - pr.eval(x, t - h)[0]) / (2 * h)
    assert np.max(np.abs(fdt - Ht)) < 1e-7 * (1 + np.max(np.abs(Ht)))


def test_eval_parameter_homotopy_interpolates_parameters():
    """F(x; p) = p0*x^2 + p1*p2*x - 1: H(x,t) uses p(t) = (1-t) p0 + t p1."""
    sys_ = inputs.TermSystem(n=1, term_eq=[0, 0, 0], term_coef=[1, 1, -1],
                             term_exp=[[2], [1], [0]],
                             term_param=[[0, -1], [1, 2], [-1, -1]], n_params=3)
    pa = np.array([1 + 1j, 2, -0.5j])
    pb = np.array([0.3, -1 + 1j, 2])
    pr = OracleProblem(sys_, kind=KIND_PARAMETER, p0=pa, p1=pb)
    x = 0.2 + 0.9j
    for t in (0.0, 0.25, 1.0):
        p = (1 - t) * pa + t * pb
        dp = pb - pa
        H, Hx, Ht = pr.eval(np.array([x]), t)
        assert abs(H[0] - (p[0] * x ** 2 + p[1] * p[2] * x - 1)) < 1e-14
        assert abs(Hx[0, 0] - (2 * p[0] * x + p[1] * p[2])) < 1e-14
        assert abs(Ht[0] - (dp[0] * x ** 2 + (dp[1] * p[2] + p[1] * dp[2]) * x)) < 1e-14


# ---------------------------------------------------------------- predictor / corrector
def test_rk4_step_is_fourth_order():
    """One RK4 step on a path known in closed form: local error ~ h^5.

    H = (1-t) g (x^2 - 1) + t (x^2 - a)  =>  x(t)^2 = ((1-t) g + t a) / ((1-t) g + t).
    An Euler step would give ratio 4, a wrong tableau weight ratio 4..16.
    """
    g, a = cmath.exp(1.3j), 2.0 - 1.0j
    sys_ = poly_system(1, [{(2,): 1.0, (0,): -a}])
    pr = OracleProblem(sys_, gamma=g)

    def xt(t):
        return cmath.sqrt(((1 - t) * g + t * a) / ((1 - t) * g + t))

    t0 = 0.3
    errs = []
    for h in (0.04, 0.02, 0.01):
        y, ok = pr.rk4_step(np.array([xt(t0)]), t0, h)
        assert ok
        errs.append(abs(y[0] - xt(t0 + h)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 25 < r1 < 40 and 25 < r2 < 40, (errs, r1, r2)


def test_newton_converges_quadratically_to_closed_form_root():
    """x^2 = a: Newton errors e_{k+1} ~ e_k^2 / (2|x|)."""
    a = 3.0 + 4.0j                        # sqrt = 2 + i
    sys_ = poly_system(1, [{(2,): 1.0, (0,): -a}])
    pr = OracleProblem(sys_)
    x = np.array([2.1 + 1.05j])
    root = 2.0 + 1.0j
    e = [abs(x[0] - root)]
    for _ in range(4):
        x, dn, ok = pr.newton_step(x, 1.0)
        assert ok
        e.append(abs(x[0] - root))
    # e_{k+1} / e_k^2 -> 1 / (2 |root|) for the first three steps, then rounding
    for k in range(3):
        assert abs(e[k + 1] / e[k] ** 2 * 2 * abs(root) - 1) < 0.2, e
    assert e[4] < 1e-15


# ---------------------------------------------------------------- whole tracker
@pytest.mark.parametrize("d,seed", [(2, 0), (5, 1), (9, 2), (14, 3), (20, 4)])
def test_univariate_roots_match_companion_matrix(d, seed):
    """n = 1: HC endpoints = eigenvalues of the companion matrix (numpy.roots)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(d + 1) + 1j * rng.standard_normal(d + 1)   # c[k] * x^k
    sys_ = poly_system(1, [{(k,): c[k] for k in range(d + 1)}])
    pr = OracleProblem(sys_, gamma=inputs.unit_gamma(seed))
    r = pr.track(threads=4)
    assert oracle.status_counts(r["status"])["finite"] == d
    want = np.roots(c[::-1]).reshape(-1, 1)
    ok, msg = same_set(r["x"], want, TOL)
    assert ok, msg


@pytest.mark.parametrize("n,d,seed", [(2, 2, 11), (3, 2, 12), (4, 2, 13), (2, 3, 14),
                                      (3, 3, 15), (6, 2, 0)])
def test_dense_random_reaches_bezout_count(n, d, seed):
    """Generic dense system: d^n distinct finite roots, each with tiny backward error."""
    sys_ = inputs.dense_system(n, d, seed)
    pr = OracleProblem(sys_, gamma=inputs.unit_gamma(seed))
    r = pr.track(threads=8)
    c = oracle.status_counts(r["status"])
    assert c["finite"] == d ** n, c
    assert distinct(r["x"], 1e-6) == d ** n
    assert np.max(r["be"]) <= 1e-10


def _newton_all_seeds(sys_, seeds, iters=60):
    """Vectorised Newton on F from many seeds (test-side evaluation of F)."""
    n = sys_.n
    ex = sys_.term_exp.astype(int)
    X = seeds.copy()
    for _ in range(iters):
        F = np.zeros((len(X), n), complex)
        J = np.zeros((len(X), n, n), complex)
        for k in range(sys_.n_terms):
            i = sys_.term_eq[k]
            c = sys_.term_coef[k]
            mono = np.prod(X ** ex[k], axis=1)
            F[:, i] += c * mono
            for j in range(n):
                if ex[k, j]:
                    e2 = ex[k].copy()
                    e2[j] -= 1
                    J[:, i, j] += c * ex[k, j] * np.prod(X ** e2, axis=1)
        with np.errstate(all="ignore"):
            X = X - np.linalg.solve(J, F[..., None])[..., 0]
    ok = np.all(np.isfinite(X), axis=1) & (np.max(np.abs(X), axis=1) < 1e6)
    X = X[ok]
    F = np.zeros((len(X), n), complex)
    for k in range(sys_.n_terms):
        F[:, sys_.term_eq[k]] += sys_.term_coef[k] * np.prod(X ** ex[k], axis=1)
    return X[np.max(np.abs(F), axis=1) < 1e-9]


@pytest.mark.parametrize("n,seed", [(2, 21), (3, 22)])
def test_bruteforce_newton_finds_the_same_root_set(n, seed):
    """Newton from 10^4 random seeds: its distinct roots = the HC endpoint set."""
    sys_ = inputs.dense_system(n, 2, seed)
    pr = OracleProblem(sys_, gamma=inputs.unit_gamma(seed))
    r = pr.track(threads=8)
    rng = np.random.default_rng(seed)
    seeds = 2.0 * (rng.standard_normal((10000, n)) + 1j * rng.standard_normal((10000, n)))
    X = _newton_all_seeds(sys_, seeds)
    reps = []
    for x in X:
        if not any(np.max(np.abs(x - y)) / max(1, np.max(np.abs(y))) < 1e-7 for y in reps):
            reps.append(x)
    ok, msg = same_set(r["x"], np.array(reps), 1e-9)
    assert ok, msg


def test_decoupled_squares_closed_form_and_real_bit():
    """x_i^2 = a_i: roots are all sign choices of sqrt(a_i); real iff a_i > 0."""
    a = [2.0, 0.5, 3.0]
    sys_ = poly_system(3, [{(2, 0, 0): 1, (0, 0, 0): -a[0]}, {(0, 2, 0): 1, (0, 0, 0): -a[1]},
                           {(0, 0, 2): 1, (0, 0, 0): -a[2]}])
    pr = OracleProblem(sys_, gamma=inputs.unit_gamma(5))
    r = pr.track()
    want = np.array([[s0 * math.sqrt(a[0]), s1 * math.sqrt(a[1]), s2 * math.sqrt(a[2])]
                     for s0, s1, s2 in itertools.product((1, -1), repeat=3)], complex)
    ok, msg = same_set(r["x"], want, TOL)
    assert ok, msg
    c = oracle.status_counts(r["status"])
    assert c["finite"] == 8 and c["real"] == 8
    # complex a: no real roots
    sys2 = poly_system(1, [{(2,): 1, (0,): -(1 + 1j)}])
    r2 = OracleProblem(sys2, gamma=inputs.unit_gamma(6)).track()
    assert oracle.status_counts(r2["status"]) == dict(finite=2, real=0, diverged=0,
                                                      singular=0, failed=0)


def test_triangular_system_closed_form():
    """x1^2 = a, x2^2 = x1 + b: x1 = +-sqrt(a), x2 = +-sqrt(x1 + b)."""
    a, b = 1.5 - 0.5j, 0.25 + 2j
    sys_ = poly_system(2, [{(2, 0): 1, (0, 0): -a}, {(0, 2): 1, (1, 0): -1, (0, 0): -b}])
    r = OracleProblem(sys_, gamma=inputs.unit_gamma(8)).track()
    want = []
    for s1 in (1, -1):
        x1 = s1 * cmath.sqrt(a)
        for s2 in (1, -1):
            want.append([x1, s2 * cmath.sqrt(x1 + b)])
    ok, msg = same_set(r["x"], np.array(want), TOL)
    assert ok, msg


def test_deficient_system_paths_to_infinity_are_not_finite():
    """x1 x2 = 1, x1 x2 + x1 = 2: one finite root (1, 1); 3 of 4 paths diverge."""
    sys_ = poly_system(2, [{(1, 1): 1, (0, 0): -1}, {(1, 1): 1, (1, 0): 1, (0, 0): -2}])
    r = OracleProblem(sys_, gamma=inputs.unit_gamma(9)).track()
    c = oracle.status_counts(r["status"])
    assert c["finite"] == 1
    fin = r["x"][(r["status"] & 0x7F) == oracle.FINITE]
    assert np.max(np.abs(fin - np.array([1, 1]))) < 1e-12


def test_double_root_is_not_classified_finite():
    """x^2 = 0: both paths end at the double root 0, which is singular."""
    sys_ = poly_system(1, [{(2,): 1.0}])
    r = OracleProblem(sys_, gamma=inputs.unit_gamma(10)).track()
    assert oracle.status_counts(r["status"])["finite"] == 0


def test_parameter_homotopy_closed_form():
    """x_i^2 = p_i: from the roots at p0 to the roots at p1 (start set given)."""
    n = 2
    sys_ = inputs.TermSystem(n=n, term_eq=[0, 0, 1, 1], term_coef=[1, -1, 1, -1],
                             term_exp=[[2, 0], [0, 0], [0, 2], [0, 0]],
                             term_param=[[-1], [0], [-1], [1]], n_params=2)
    p0 = inputs.random_complex(2, 31)
    p1 = np.array([4.0 + 0j, -1.0 + 0j])
    start = np.array([[s0 * np.sqrt(p0[0]), s1 * np.sqrt(p0[1])]
                      for s0 in (1, -1) for s1 in (1, -1)])
    r = OracleProblem(sys_, kind=KIND_PARAMETER, p0=p0, p1=p1).track(start=start)
    want = np.array([[s0 * 2.0, s1 * 1j] for s0 in (1, -1) for s1 in (1, -1)])
    ok, msg = same_set(r["x"], want, TOL)
    assert ok, msg


def test_track_is_deterministic_across_thread_counts():
    sys_ = inputs.dense_system(4, 2, 40)
    pr = OracleProblem(sys_, gamma=inputs.unit_gamma(40))
    a = pr.track(threads=1)
    b = pr.track(threads=8)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["status"], b["status"])


# ---------------------------------------------------------------- classification quantities
def test_backward_error_closed_form_values():
    """Hand-computed backward errors max_i |F_i(x)| / sum_k |c_k| |x^a_k|.

    F = (1+i) x - 2 at x = 1: |F| = |-1+i| = sqrt 2, denominator
    |1+i| * 1 + |-2| = sqrt 2 + 2.  Dropping the |c| factor would give
    sqrt 2 / 3; returning 0 or omitting the constant term fails too."""
    pr = OracleProblem(poly_system(1, [{(1,): 1 + 1j, (0,): -2.0}]))
    be = pr.backward_error(np.array([1.0 + 0j]))
    assert abs(be - math.sqrt(2) / (math.sqrt(2) + 2)) < 1e-15
    # x^2 - 4 at x = 2 + delta: |4 delta + delta^2| / ((2 + delta)^2 + 4)
    pr = OracleProblem(poly_system(1, [{(2,): 1.0, (0,): -4.0}]))
    for delta in (1e-3, -2e-5j, 0.5 + 0.25j):
        x = 2 + delta
        want = abs(4 * delta + delta ** 2) / (abs(x) ** 2 + 4)
        # F is formed with cancellation: its rounding is a few ulps of the
        # denominator, so the bound is absolute
        assert abs(pr.backward_error(np.array([x])) - want) <= 1e-15
    # the maximum over equations, each scaled by its own terms (point (1, 3)):
    # F1 = x1 - 1 -> 0; F2 = 2 x1 x2 - 5 -> 1 / (6 + 5)
    pr = OracleProblem(poly_system(2, [{(1, 0): 1.0, (0, 0): -1.0},
                                       {(1, 1): 2.0, (0, 0): -5.0}]))
    assert abs(pr.backward_error(np.array([1.0, 3.0 + 0j])) - 1 / 11) < 1e-15
    # and exactly zero at the exact root
    assert pr.backward_error(np.array([1.0, 2.5 + 0j])) == 0.0


def _linear_system(A, b):
    """F(x) = A x - b as a term list (its Jacobian is A everywhere)."""
    n = A.shape[0]
    polys = []
    for i in range(n):
        poly = {(0,) * n: -b[i]}
        for j in range(n):
            if A[i, j] != 0:
                e = [0] * n
                e[j] = 1
                poly[tuple(e)] = A[i, j]
        polys.append(poly)
    return poly_system(n, polys)


def test_cond1_closed_form_values():
    """cond_1(A) = ||A||_1 ||A^-1||_1 with the modulus of complex entries.

    diag(3+4i, 1): 5 * 1 = 5 (|Re| + |Im| would give 7).  The lower
    triangular L = [[1,0,0],[0,10,0],[50,0,100]] has column sums 51, 10, 100
    and L^-1 = [[1,0,0],[0,0.1,0],[-0.5,0,0.01]] column sums 1.5, 0.1, 0.01:
    cond_1 = 150 (an inverse left out gives 100).  For U below the 1-norm
    and the infinity-norm condition numbers differ, so a transposed norm
    fails there."""
    A = np.diag([3 + 4j, 1.0])
    pr = OracleProblem(_linear_system(A, np.ones(2)))
    assert abs(pr.cond1(np.zeros(2, complex)) - 5.0) < 1e-14
    L = np.array([[1, 0, 0], [0, 10, 0], [50, 0, 100]], complex)
    for M, want in ((L, 150.0), (L.T, 150.0)):
        pr = OracleProblem(_linear_system(M, np.ones(3)))
        assert abs(pr.cond1(np.zeros(3, complex)) - want) < 1e-12
    U = np.array([[2, 7, 0], [0, 1, 3], [0, 0, 4]], complex)
    pr = OracleProblem(_linear_system(U, np.ones(3)))
    want = np.linalg.norm(U, 1) * np.linalg.norm(np.linalg.inv(U), 1)
    assert abs(pr.cond1(np.zeros(3, complex)) - want) < 1e-12 * want
    assert abs(want - np.linalg.norm(U, np.inf) * np.linalg.norm(np.linalg.inv(U), np.inf)) > 1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cond1_matches_library_on_random_jacobians(seed):
    """At a random point of a dense quadratic system, cond_1(dF/dx) equals
    numpy's 1-norm condition number of the oracle's own Jacobian (the
    Jacobian itself is pinned by finite differences above)."""
    sys_ = inputs.dense_system(4, 2, seed)
    pr = OracleProblem(sys_)
    x = inputs.random_complex(4, seed + 50)
    _, Hx, _ = pr.eval(x, 1.0)
    assert abs(pr.cond1(x) - np.linalg.cond(Hx, 1)) <= 1e-10 * np.linalg.cond(Hx, 1)


# ---------------------------------------------------------------- coefficient interpolation
def test_coefficient_interpolation_closed_form():
    """Sec. 6 interpolates the coefficients: F = p0 p1 x^2 - 1 with p(0) = (a0,
    b0), p(1) = (a1, b1) gives H = c(t) x^2 - 1, c(t) = (1-t) a0 b0 + t a1 b1,
    dH/dt = (a1 b1 - a0 b0) x^2, dH/dx = 2 c(t) x; the parameter homotopy
    instead has c(t) = ((1-t) a0 + t a1)((1-t) b0 + t b1)."""
    sys_ = inputs.TermSystem(n=1, term_eq=np.array([0, 0]), term_coef=np.array([1.0, -1.0]),
                             term_exp=np.array([[2], [0]]), term_param=np.array([[0, 1], [-1, -1]]),
                             n_params=2)
    a0, b0, a1, b1 = 1 + 2j, 0.5 - 1j, -2 + 0.25j, 3 + 1j
    p0, p1 = np.array([a0, b0]), np.array([a1, b1])
    x, t = np.array([0.7 - 0.4j]), 0.3
    pc = OracleProblem(sys_, kind=oracle.KIND_COEFFICIENT, p0=p0, p1=p1)
    H, Hx, Ht = pc.eval(x, t)
    c = (1 - t) * a0 * b0 + t * a1 * b1
    assert abs(H[0] - (c * x[0] ** 2 - 1)) < 1e-14
    assert abs(Ht[0] - (a1 * b1 - a0 * b0) * x[0] ** 2) < 1e-14
    assert abs(Hx[0, 0] - 2 * c * x[0]) < 1e-14
    pp = OracleProblem(sys_, kind=oracle.KIND_PARAMETER, p0=p0, p1=p1)
    cp = ((1 - t) * a0 + t * a1) * ((1 - t) * b0 + t * b1)
    assert abs(pp.eval(x, t)[0][0] - (cp * x[0] ** 2 - 1)) < 1e-14
    # tracking from x = 1/sqrt(a0 b0) ends at a square root of 1/(a1 b1)
    r = pc.track(start=np.array([[1 / np.sqrt(a0 * b0)]]))
    assert (r["status"][0] & 0x7F) == oracle.FINITE
    assert abs(r["x"][0, 0] ** 2 * a1 * b1 - 1) < 1e-12


def test_coefficient_interpolation_equals_parameter_homotopy_when_linear():
    """When every coefficient is one parameter (the dense family written as
    a parameter family), interpolating coefficients and interpolating
    parameters are the same homotopy: identical results, bit for bit."""
    sys_, p1, p0 = inputs.dense_parameter_family(3, 2, 62)
    start = np.array([OracleProblem(inputs.dense_system(3, 2, 62)).start_point(k) for k in range(8)])
    a = OracleProblem(sys_, kind=KIND_PARAMETER, p0=p0, p1=p1).track(start=start)
    b = OracleProblem(sys_, kind=oracle.KIND_COEFFICIENT, p0=p0, p1=p1).track(start=start)
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["x"], b["x"])


# ---------------------------------------------------------------- power-series endgame
def _triple_root_system():
    """(x1 - 1)^3 = 0, x2 = 1: one root (1, 1) of multiplicity 3, reached by
    all three total-degree paths with cycle number 3."""
    return poly_system(2, [{(3, 0): 1.0, (2, 0): -3.0, (1, 0): 3.0, (0, 0): -1.0},
                           {(0, 1): 1.0, (0, 0): -1.0}])


def test_endgame_finds_the_multiple_root():
    """Closed form: every path of the triple root ends within 1e-8 of (1, 1);
    those the endgame finishes are classified singular (cycle number 3 > 1),
    where without it the same paths fail by step-size underflow."""
    sys_ = _triple_root_system()
    off = OracleProblem(sys_, gamma=inputs.unit_gamma(4)).track()
    on = OracleProblem(sys_, gamma=inputs.unit_gamma(4)).track(settings=dict(endgame=1))
    assert np.all((off["status"] & 0x7F) == oracle.FAIL_STEP)
    sing = (on["status"] & 0x7F) == oracle.SINGULAR
    assert sing.sum() >= 2
    assert np.max(np.abs(on["x"][sing] - np.array([1.0, 1.0]))) < 1e-8
    assert np.all(on["be"][sing] <= 1e-10)
    steps_on = on["counts"][sing, :2].sum()
    steps_off = off["counts"][sing, :2].sum()
    assert steps_on < steps_off


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_endgame_leaves_nonsingular_endpoints_alone(seed):
    """Dense random systems (all roots simple): the endgame's predictions
    converge with cycle number 1, and refinement gives the same statuses and
    endpoints as without it."""
    sys_ = inputs.dense_system(4, 2, seed)
    a = OracleProblem(sys_, gamma=inputs.unit_gamma(seed)).track()
    b = OracleProblem(sys_, gamma=inputs.unit_gamma(seed)).track(settings=dict(endgame=1))
    assert np.array_equal(a["status"], b["status"])
    ok, msg = same_set(a["x"], b["x"], 1e-10)
    assert ok, msg


def test_endgame_makes_no_prediction_for_paths_to_infinity():
    """x1 x2 = 1, x1 x2 + x1 = 2: one finite root (1, 1).  Paths to infinity
    have growing sample differences, so the endgame predicts nothing for
    them: no path other than the one to (1, 1) ends finite (a prediction
    refined onto (1, 1) would be a path jump)."""
    sys_ = poly_system(2, [{(1, 1): 1, (0, 0): -1}, {(1, 1): 1, (1, 0): 1, (0, 0): -2}])
    r = OracleProblem(sys_, gamma=inputs.unit_gamma(9)).track(settings=dict(endgame=1))
    assert oracle.status_counts(r["status"])["finite"] == 1


def test_oracle_jacobian_matches_the_paper_term_tuples():
    """Sec. 6 worked example: the oracle's dH/dx entries (1,1) and (2,1) of
    the example family equal the paper's printed tuple representations of A
    and B evaluated at a(t) = (1 - t) a(0) + t a(1) (x3 = 1), at random
    points; and the tuple padded with s = 0 adds nothing."""
    import sec6_example as ex
    tup = ex.tuples()
    fam = ex.family()
    p0, p1 = ex.parameters(1)
    op = OracleProblem(fam, kind=KIND_PARAMETER, p0=p0, p1=p1)
    rng = np.random.default_rng(7)
    for _ in range(5):
        x = rng.normal(size=2) + 1j * rng.normal(size=2)
        t = float(rng.uniform())
        a = (1 - t) * p0 + t * p1
        _, Hx, _ = op.eval(x, t)
        A = ex.tuple_value(tup["A"], a, x)
        B = ex.tuple_value(tup["B"], a, x)
        assert abs(Hx[0, 0] - A) <= 1e-13 * (1 + abs(A)), (Hx[0, 0], A)
        assert abs(Hx[1, 0] - B) <= 1e-13 * (1 + abs(B)), (Hx[1, 0], B)
        assert ex.tuple_value(tup["B"][2:], a, x) == 0

"""Seeded synthetic inputs for the homotopy-continuation tracker.

This module produces *problem data only*: polynomial systems as term lists
(equation index, complex coefficient, exponent vector, parameter factors),
the random homotopy constant gamma, and target parameter vectors.  It holds
none of the method's arithmetic (no evaluation, no solve, no tracking), so
both the CUDA path and the CPU oracle may consume what it produces.

Term-list format (shared by the C-ABI and the oracle):
  term_eq    int32   [T]          equation index of each term
  term_coef  complex [T]          scalar coefficient s_k
  term_exp   uint8   [T, n]       exponent vector alpha_k of the monomial x^alpha
  term_param int32   [T, maxpf]   parameter indices multiplied into the
                                  coefficient (-1 = no factor); maxpf may be 0

A term's value is s_k * prod_l p_{param_kl} * x^{alpha_k}.  The paper's
target systems F(x) (Sec. 3, Eq. 1) are sums of such terms; the library
derives its evaluation tables (Sec. 6) from this list.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class TermSystem:
    """A square polynomial system F(x; p) in term-list form."""

    n: int
    term_eq: np.ndarray          # int32 [T]
    term_coef: np.ndarray        # complex128 [T]
    term_exp: np.ndarray         # uint8 [T, n]
    term_param: np.ndarray = field(default=None)  # int32 [T, maxpf] or None
    n_params: int = 0
    name: str = ""

    def __post_init__(self):
        self.term_eq = np.ascontiguousarray(self.term_eq, dtype=np.int32)
        self.term_coef = np.ascontiguousarray(self.term_coef, dtype=np.complex128)
        self.term_exp = np.ascontiguousarray(self.term_exp, dtype=np.uint8).reshape(-1, self.n)
        if self.term_param is None:
            self.term_param = np.zeros((len(self.term_eq), 0), dtype=np.int32)
        self.term_param = np.ascontiguousarray(self.term_param, dtype=np.int32)

    @property
    def n_terms(self) -> int:
        return int(self.term_eq.shape[0])

    @property
    def max_pfac(self) -> int:
        return int(self.term_param.shape[1])

    def degrees(self) -> np.ndarray:
        """Total degree of each equation (max over its terms)."""
        deg = np.zeros(self.n, dtype=np.int64)
        tot = self.term_exp.astype(np.int64).sum(axis=1)
        np.maximum.at(deg, self.term_eq, tot)
        return deg


def monomials(n: int, d: int) -> np.ndarray:
    """Exponent vectors of all monomials of degree <= d in n variables.

    Graded order: degree 0 first, then degree 1, ...; inside a degree,
    lexicographic on the sorted variable-index tuple.  Count C(n+d, d).
    """
    rows = []
    for deg in range(d + 1):
        for combo in itertools.combinations_with_replacement(range(n), deg):
            e = np.zeros(n, dtype=np.uint8)
            for v in combo:
                e[v] += 1
            rows.append(e)
    return np.array(rows, dtype=np.uint8).reshape(-1, n)


def unit_gamma(seed: int) -> complex:
    """Random unit-modulus constant gamma = exp(i*theta), theta ~ U[0, 2pi)."""
    rng = np.random.default_rng([seed, 0x6A])
    theta = rng.uniform(0.0, 2.0 * math.pi)
    return complex(math.cos(theta), math.sin(theta))


def dense_coefficients(n: int, d: int, seed: int) -> np.ndarray:
    """Coefficients [n, M] with re, im ~ N(0, 1) iid, for the monomials(n, d) order."""
    rng = np.random.default_rng([seed, n, d])
    m = math.comb(n + d, d)
    return rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))


def dense_system(n: int, d: int, seed: int) -> TermSystem:
    """Dense random system: every monomial of degree <= d in every equation.

    This is the workload that stands in for the paper's polynomial benchmarks
    (Table 1): n equations of degree d, coefficients complex Gaussian.
    """
    exps = monomials(n, d)
    coef = dense_coefficients(n, d, seed)
    m = exps.shape[0]
    term_eq = np.repeat(np.arange(n, dtype=np.int32), m)
    term_exp = np.tile(exps, (n, 1))
    return TermSystem(n=n, term_eq=term_eq, term_coef=coef.reshape(-1),
                      term_exp=term_exp, name=f"dense_n{n}_d{d}_s{seed}")


def dense_batch(n: int, d: int, seeds) -> tuple[TermSystem, np.ndarray]:
    """One term-list structure plus per-instance coefficient vectors [I, T]."""
    base = dense_system(n, d, seeds[0])
    coefs = np.stack([dense_coefficients(n, d, s).reshape(-1) for s in seeds])
    return base, coefs


def system_from_polys(n: int, polys) -> TermSystem:
    """Build a TermSystem from a list (one per equation) of {exponent tuple: coef}."""
    eqs, cf, ex = [], [], []
    for i, poly in enumerate(polys):
        for e, c in poly.items():
            eqs.append(i)
            cf.append(complex(c))
            ex.append(np.array(e, dtype=np.uint8))
    return TermSystem(n=n, term_eq=np.array(eqs), term_coef=np.array(cf),
                      term_exp=np.array(ex).reshape(-1, n))


def random_complex(shape, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------------------
# Parameter-homotopy problem families (paper Sec. 4, configs with synthetic
# scenes).  Polynomials are built as dicts {(x-exponent tuple, sorted param
# index tuple): coefficient}; this is the problem statement written out as
# data, not part of the method.
# ---------------------------------------------------------------------------

class _Poly:
    """Polynomial in unknowns x (n) whose coefficients are monomials in params."""

    __slots__ = ("n", "t")

    def __init__(self, n, terms=None):
        self.n = n
        self.t = dict(terms or {})

    @staticmethod
    def const(n, c):
        return _Poly(n, {((0,) * n, ()): complex(c)})

    @staticmethod
    def var(n, j, c=1.0):
        e = [0] * n
        e[j] = 1
        return _Poly(n, {(tuple(e), ()): complex(c)})

    @staticmethod
    def param(n, l, c=1.0):
        return _Poly(n, {((0,) * n, (l,)): complex(c)})

    def __add__(self, o):
        if not isinstance(o, _Poly):
            o = _Poly.const(self.n, o)
        t = dict(self.t)
        for k, v in o.t.items():
            t[k] = t.get(k, 0) + v
        return _Poly(self.n, {k: v for k, v in t.items() if v != 0})

    __radd__ = __add__

    def __neg__(self):
        return _Poly(self.n, {k: -v for k, v in self.t.items()})

    def __sub__(self, o):
        return self + (-o if isinstance(o, _Poly) else -complex(o))

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not isinstance(o, _Poly):
            return _Poly(self.n, {k: v * o for k, v in self.t.items() if v * o != 0})
        t = {}
        for (e1, p1), c1 in self.t.items():
            for (e2, p2), c2 in o.t.items():
                k = (tuple(a + b for a, b in zip(e1, e2)), tuple(sorted(p1 + p2)))
                t[k] = t.get(k, 0) + c1 * c2
        return _Poly(self.n, {k: v for k, v in t.items() if v != 0})

    __rmul__ = __mul__


def _system_from(n, n_params, polys, name):
    eqs, cf, ex, pa = [], [], [], []
    maxpf = max((len(p) for poly in polys for (_, p) in poly.t), default=0)
    for i, poly in enumerate(polys):
        for (e, p), c in sorted(poly.t.items()):
            eqs.append(i)
            cf.append(c)
            ex.append(e)
            pa.append(list(p) + [-1] * (maxpf - len(p)))
    return TermSystem(n=n, term_eq=np.array(eqs), term_coef=np.array(cf),
                      term_exp=np.array(ex, dtype=np.uint8).reshape(-1, n),
                      term_param=np.array(pa, dtype=np.int32).reshape(-1, maxpf),
                      n_params=n_params, name=name)


@dataclass
class ParamFamily:
    """A parameter-homotopy problem family F(x; p)."""

    system: TermSystem
    unknowns: list            # names of the unknowns, in order
    params: list              # names of the parameters, in order
    linear_params: list       # indices of params in which F is affine (for seeding)
    unit_groups: list         # unknown-index groups constrained by q.q = 1
    name: str
    # optional: (x0, p) -> x0 with the equations that involve no linear
    # parameter satisfied (monodromy seeding); None when there are none
    complete_seed: object = None
    # sign symmetries (bit masks of unknowns whose negation maps solutions to
    # solutions); None: one per unit-quaternion group
    sym_masks: list = None

    @property
    def sign_masks(self) -> list:
        """Bit masks of the sign symmetries: by default the unit-quaternion
        groups (R(q) is quadratic in q, so negating a group maps solutions to
        solutions)."""
        if self.sym_masks is not None:
            return list(self.sym_masks)
        return [sum(1 << j for j in grp) for grp in self.unit_groups]


def triangulation_family(views: int = 4) -> ParamFamily:
    """N-view optimal triangulation by Lagrange multipliers (paper Sec. 4).

    Unknowns: image corrections (u_k, v_k), k = 1..N, and one multiplier
    lambda_ij per view pair i < j: 2N + N(N-1)/2 unknowns (14 for N = 4).
    Parameters: normalised image points (xi_k, eta_k) and the nine entries of
    each pairwise essential matrix E_ij (row-major): 2N + 9 N(N-1)/2 (62).
    With g_k = (xi_k - u_k, eta_k - v_k, 1) the Lagrangian is
      sum_k (u_k^2 + v_k^2) + sum_{i<j} lambda_ij g_j^T E_ij g_i
    and the equations are its derivatives (all quadratic):
      2 u_k - sum_{i<k} l_ik e1^T E_ik g_i - sum_{j>k} l_kj g_j^T E_kj e1 = 0
      2 v_k - (same with e2) = 0
      g_j^T E_ij g_i = 0.
    """
    N = views
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    n = 2 * N + len(pairs)
    P = 2 * N + 9 * len(pairs)
    U = lambda k: 2 * k
    V = lambda k: 2 * k + 1
    LAM = {pr: 2 * N + a for a, pr in enumerate(pairs)}
    XI = lambda k: 2 * k
    ETA = lambda k: 2 * k + 1
    EP = {pr: 2 * N + 9 * a for a, pr in enumerate(pairs)}

    def g(k):
        return [_Poly.param(n, XI(k)) - _Poly.var(n, U(k)),
                _Poly.param(n, ETA(k)) - _Poly.var(n, V(k)),
                _Poly.const(n, 1.0)]

    def E(pr, a, b):
        return _Poly.param(n, EP[pr] + 3 * a + b)

    def bil(pr, left, right):  # left^T E_pr right
        out = _Poly(n)
        for a in range(3):
            for b in range(3):
                out = out + left[a] * E(pr, a, b) * right[b]
        return out

    unit = [[_Poly.const(n, 1.0), _Poly(n), _Poly(n)], [_Poly(n), _Poly.const(n, 1.0), _Poly(n)]]
    polys = []
    for k in range(N):
        for c, var in ((0, U), (1, V)):
            eq = _Poly.var(n, var(k), 2.0)
            for (i, j) in pairs:
                lam = _Poly.var(n, LAM[(i, j)])
                if j == k:     # d/du_j of g_j^T E g_i = -e^T E g_i
                    eq = eq - lam * bil((i, j), unit[c], g(i))
                elif i == k:   # d/du_i of g_j^T E g_i = -g_j^T E e
                    eq = eq - lam * bil((i, j), g(j), [unit[c][0], unit[c][1], unit[c][2]])
            polys.append(eq)
    for pr in pairs:
        polys.append(bil(pr, g(pr[1]), g(pr[0])))
    unknowns = [f"{s}{k + 1}" for k in range(N) for s in ("u", "v")] + \
               [f"l{i + 1}{j + 1}" for (i, j) in pairs]
    params = [f"{s}{k + 1}" for k in range(N) for s in ("xi", "eta")] + \
             [f"E{i + 1}{j + 1}_{a}{b}" for (i, j) in pairs for a in range(3) for b in range(3)]
    return ParamFamily(system=_system_from(n, P, polys, f"triangulation{N}"), unknowns=unknowns,
                       params=params, linear_params=list(range(2 * N, P)), unit_groups=[],
                       name=f"triangulation{N}")


def _quat_rot(q):
    """Rotation matrix (list of lists of _Poly) of an unnormalised quaternion (q0, q1, q2, q3)."""
    q0, q1, q2, q3 = q
    return [[q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3), 2 * (q1 * q3 + q0 * q2)],
            [2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, 2 * (q2 * q3 - q0 * q1)],
            [2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1), q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3]]


def trifocal_family() -> ParamFamily:
    """Trifocal relative pose with a shared unknown focal length (paper Sec. 4).

    Unknowns (18): phi (= s/f, pixel coordinates pre-scaled by s), the
    quaternions q12, q13 of R_12, R_13, T_12 = (a, b, 1) (affine chart fixing
    the scale), T_13 (3), and the depths rho_p of the four points in view 1.
    Parameters (24): image coordinates (xi_vp, eta_vp) of point p in view v,
    principal point subtracted and divided by s.  With
      w = rho_p R(q_1v) (phi xi_1p, phi eta_1p, 1)^T + T_1v
    the depth in view v is w_3 and the equations are
      phi xi_vp w_3 - w_1 = 0,  phi eta_vp w_3 - w_2 = 0   (v = 2, 3; 16 equations)
      q12 . q12 - 1 = 0,  q13 . q13 - 1 = 0.
    """
    n, P = 18, 24
    PHI, Q12, Q13, AB, T13, RHO = 0, 1, 5, 9, 11, 14
    X = lambda j: _Poly.var(n, j)
    PXI = lambda v, p: _Poly.param(n, 2 * (3 * p + v))       # view v = 0, 1, 2
    PETA = lambda v, p: _Poly.param(n, 2 * (3 * p + v) + 1)
    phi = X(PHI)
    polys = []
    for v, qb in ((1, Q12), (2, Q13)):
        R = _quat_rot([X(qb + a) for a in range(4)])
        T = [X(AB), X(AB + 1), _Poly.const(n, 1.0)] if v == 1 else [X(T13 + a) for a in range(3)]
        for p in range(4):
            g1 = [phi * PXI(0, p), phi * PETA(0, p), _Poly.const(n, 1.0)]
            w = []
            for a in range(3):
                acc = T[a]
                for b in range(3):
                    acc = acc + X(RHO + p) * R[a][b] * g1[b]
                w.append(acc)
            polys.append(phi * PXI(v, p) * w[2] - w[0])
            polys.append(phi * PETA(v, p) * w[2] - w[1])
    for qb in (Q12, Q13):
        polys.append(sum((X(qb + a) * X(qb + a) for a in range(4)), _Poly(n)) - 1.0)
    unknowns = ["phi"] + [f"q12_{a}" for a in range(4)] + [f"q13_{a}" for a in range(4)] + \
               ["a", "b"] + [f"T13_{a}" for a in range(3)] + [f"rho{p + 1}" for p in range(4)]
    params = [f"{s}{v + 1}_{p + 1}" for p in range(4) for v in range(3) for s in ("xi", "eta")]
    linear = [2 * (3 * p + v) + c for p in range(4) for v in (1, 2) for c in (0, 1)]
    return ParamFamily(system=_system_from(n, P, polys, "trifocal_f"), unknowns=unknowns,
                       params=params, linear_params=sorted(linear),
                       unit_groups=[list(range(Q12, Q12 + 4)), list(range(Q13, Q13 + 4))],
                       name="trifocal_f")


def p3p_family() -> ParamFamily:
    """P3P in the depths (paper Sec. 4, Eq. P3PafterElim): with image points
    gamma_k = (xi_k, eta_k, 1) and depths rho_k, the 3D points are
    rho_k gamma_k in the camera frame, and the camera-independent distances
    of the world points fix
      |rho2 g2 - rho1 g1|^2 = a,  |rho3 g3 - rho1 g1|^2 = b,
      (rho2 g2 - rho1 g1) . (rho3 g3 - rho1 g1) = c,
    a = |G2 - G1|^2, b = |G3 - G1|^2, c = (G2 - G1) . (G3 - G1).
    Unknowns rho1..3; parameters (xi_k, eta_k) k = 1..3, then a, b, c.  Every
    term has even degree in the depths (rho -> -rho maps solutions to
    solutions: sign mask 0b111); Bezout and the generic count are 8."""
    n, P = 3, 9
    rho = [_Poly.var(n, k) for k in range(3)]
    g = [[_Poly.param(n, 2 * k), _Poly.param(n, 2 * k + 1), _Poly.const(n, 1.0)] for k in range(3)]

    def diff(i, j):   # rho_i g_i - rho_j g_j
        return [rho[i] * g[i][a] - rho[j] * g[j][a] for a in range(3)]

    def dot(u, v):
        out = _Poly(n)
        for a in range(3):
            out = out + u[a] * v[a]
        return out
    d21, d31 = diff(1, 0), diff(2, 0)
    polys = [dot(d21, d21) - _Poly.param(n, 6), dot(d31, d31) - _Poly.param(n, 7),
             dot(d21, d31) - _Poly.param(n, 8)]
    params = [f"{s}{k + 1}" for k in range(3) for s in ("xi", "eta")] + ["a", "b", "c"]
    return ParamFamily(system=_system_from(n, P, polys, "p3p"),
                       unknowns=["rho1", "rho2", "rho3"], params=params,
                       linear_params=[6, 7, 8], unit_groups=[], name="p3p", sym_masks=[0b111])


def pose5_depth_family() -> ParamFamily:
    """Relative pose with depth reconstruction from five points (paper Sec. 4,
    Eq. FullRigidMotion): rhobar_i gbar_i = R(q) rho_i g_i + T, i = 1..5, with
    g_i = (xi_i, eta_i, 1) in view 1, gbar_i = (xibar_i, etabar_i, 1) in view
    2, the rotation by an unnormalised quaternion q with q . q = 1, and the
    translation on the chart T = (a, b, 1) (the unit direction of the paper
    fixed by its third coordinate instead, which keeps 16 unknowns for 16
    equations).  Unknowns: rho_1..5, rhobar_1..5, q_0..3, a, b.  Parameters:
    (xi_i, eta_i, xibar_i, etabar_i), i = 1..5.  R(q) is quadratic in q:
    negating q maps solutions to solutions (sign mask of q)."""
    n, P = 16, 20
    RHO, RBAR, Q, A = 0, 5, 10, 14
    X = lambda j: _Poly.var(n, j)
    R = _quat_rot([X(Q + a) for a in range(4)])
    T = [X(A), X(A + 1), _Poly.const(n, 1.0)]
    polys = []
    for i in range(5):
        g = [_Poly.param(n, 4 * i), _Poly.param(n, 4 * i + 1), _Poly.const(n, 1.0)]
        gb = [_Poly.param(n, 4 * i + 2), _Poly.param(n, 4 * i + 3), _Poly.const(n, 1.0)]
        for r in range(3):
            rg = _Poly(n)
            for c in range(3):
                rg = rg + R[r][c] * g[c]
            polys.append(X(RBAR + i) * gb[r] - X(RHO + i) * rg - T[r])
    polys.append(sum((X(Q + a) * X(Q + a) for a in range(4)), _Poly(n)) - 1.0)
    unknowns = [f"rho{i + 1}" for i in range(5)] + [f"rhobar{i + 1}" for i in range(5)] + \
               [f"q{a}" for a in range(4)] + ["a", "b"]
    params = [f"{s}{i + 1}" for i in range(5) for s in ("xi", "eta", "xibar", "etabar")]

    def complete(x0, p):
        # the third row of each point equation holds no parameter in which F
        # is affine: set rhobar_i = rho_i (R(q) g_i)_3 + 1
        q = x0[Q:Q + 4]
        Rq = _rot_numeric(q)
        for i in range(5):
            gi = np.array([p[4 * i], p[4 * i + 1], 1.0])
            x0[RBAR + i] = x0[RHO + i] * (Rq[2] @ gi) + 1.0
        return x0
    return ParamFamily(system=_system_from(n, P, polys, "pose5_depth"), unknowns=unknowns,
                       params=params,
                       linear_params=sorted([4 * i + 2 for i in range(5)] +
                                            [4 * i + 3 for i in range(5)]),
                       unit_groups=[list(range(Q, Q + 4))], name="pose5_depth",
                       complete_seed=complete)


def _rot_numeric(q):
    """R(q) of an unnormalised complex quaternion (the same formula as _quat_rot)."""
    q0, q1, q2, q3 = q
    return np.array([[q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3),
                      2 * (q1 * q3 + q0 * q2)],
                     [2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3,
                      2 * (q2 * q3 - q0 * q1)],
                     [2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1),
                      q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3]], dtype=np.complex128)


# ---------------------------------------------------------------- scenes
def _rot_axis_angle(axis, ang):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _quat_of(R):
    """A unit quaternion (q0, q1, q2, q3) with _quat_rot(q) = R (Shepperd's method)."""
    tr = np.trace(R)
    if tr > 0:
        s = 2.0 * np.sqrt(tr + 1.0)
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    else:
        i = int(np.argmax(np.diag(R)))
        j, k = (i + 1) % 3, (i + 2) % 3
        s = 2.0 * np.sqrt(1.0 + R[i, i] - R[j, j] - R[k, k])
        q = [0.0] * 4
        q[0] = (R[k, j] - R[j, k]) / s
        q[1 + i] = 0.25 * s
        q[1 + j] = (R[j, i] + R[i, j]) / s
        q[1 + k] = (R[k, i] + R[i, k]) / s
    return np.array(q)


def triangulation_scene(seed: int, views: int = 4, noise_px: float = 1.0, f: float = 1000.0,
                        width: int = 1920, height: int = 1080, pose_noise_deg: float = 2.0,
                        pose_noise_t: float = 0.03):
    """Synthetic N-view scene: pinhole cameras (focal f px) on the radius-5
    sphere looking at the origin, random roll, one 3D point uniform in the
    centred unit cube, projections with N(0, noise_px) pixel noise.

    Each essential matrix E_ij (g_j^T E_ij g_i = 0) comes from its own
    perturbed relative pose: rotation by N(0, pose_noise_deg) degrees about a
    random axis, translation direction perturbed by N(0, pose_noise_t).
    Pairwise-estimated essential matrices are never exactly consistent; with
    exactly consistent ones the pairwise constraints of three or more views
    are redundant at the data and the Lagrange system's optimum is a singular
    root (pose_noise_deg = pose_noise_t = 0 gives that degenerate case).

    Returns (p1, truth): p1 = parameter vector (normalised image points and
    the nine entries of each E_ij), truth = dict with the noise-free image
    points packed with the same E's (p_clean), cameras and the 3D point.
    """
    rng = np.random.default_rng([seed, 0x7A1])
    Kinv = np.linalg.inv(np.array([[f, 0, width / 2], [0, f, height / 2], [0, 0, 1.0]]))
    for _attempt in range(1000):
        X = rng.uniform(-0.5, 0.5, 3)
        Rs, ts, pix = [], [], []
        ok = True
        for _ in range(views):
            c = rng.standard_normal(3)
            c = 5.0 * c / np.linalg.norm(c)
            z = -c / np.linalg.norm(c)                       # optical axis towards the origin
            tmp = np.array([0.0, 0.0, 1.0]) if abs(z[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
            x = np.cross(tmp, z); x /= np.linalg.norm(x)
            y = np.cross(z, x)
            R = np.stack([x, y, z])                          # world -> camera
            roll = rng.uniform(0, 2 * np.pi)
            R = _rot_axis_angle([0, 0, 1], roll) @ R
            t = -R @ c
            xc = R @ X + t
            if xc[2] <= 0:
                ok = False
                break
            u = f * xc[0] / xc[2] + width / 2
            v = f * xc[1] / xc[2] + height / 2
            if not (0 <= u < width and 0 <= v < height):
                ok = False
                break
            Rs.append(R); ts.append(t); pix.append((u, v))
        if ok:
            break
    pairs = [(i, j) for i in range(views) for j in range(i + 1, views)]
    Es = []
    for (i, j) in pairs:
        Rij = Rs[j] @ Rs[i].T
        tij = ts[j] - Rij @ ts[i]
        if pose_noise_deg > 0:
            Rij = _rot_axis_angle(rng.standard_normal(3),
                                  np.deg2rad(rng.normal(0, pose_noise_deg))) @ Rij
        if pose_noise_t > 0:
            nrm = np.linalg.norm(tij)
            tij = tij / nrm + rng.normal(0, pose_noise_t, 3)
            tij = tij / np.linalg.norm(tij) * nrm
        tx = np.array([[0, -tij[2], tij[1]], [tij[2], 0, -tij[0]], [-tij[1], tij[0], 0]])
        Es.append(tx @ Rij)

    def pack(pixels):
        pts = []
        for (u, v) in pixels:
            g = Kinv @ np.array([u, v, 1.0])
            pts += [g[0], g[1]]
        return np.array(pts + [e for E in Es for e in E.reshape(-1)], dtype=np.complex128)

    noisy = [(u + rng.normal(0, noise_px), v + rng.normal(0, noise_px)) for (u, v) in pix]
    return pack(noisy), dict(p_clean=pack(pix), R=Rs, t=ts, X=X, pixels=pix, f=f)


def trifocal_scene(seed: int, noise_px: float = 0.5, width: int = 1920, height: int = 1080,
                   scale: float = 1000.0):
    """Synthetic three-view scene for the trifocal family: f ~ U[500, 2000] px
    shared by the three cameras, camera 1 at the identity, R_12, R_13 about a
    random axis by U[0, 30] degrees, T_1v of random direction and length
    U[0.5, 1.5], four points with pixel position uniform in image 1 and depth
    U[2, 10], visible in all views; N(0, noise_px) pixel noise.

    Returns (p1, truth): truth has p_clean and the ground-truth unknowns
    x_true in the family's chart (T_12 scaled to (a, b, 1)).
    """
    rng = np.random.default_rng([seed, 0x7F1])
    for _attempt in range(1000):
        f = rng.uniform(500, 2000)
        Rv, Tv = [np.eye(3)], [np.zeros(3)]
        for _ in range(2):
            ax = rng.standard_normal(3)
            Rv.append(_rot_axis_angle(ax, np.deg2rad(rng.uniform(0, 30))))
            d = rng.standard_normal(3)
            Tv.append(d / np.linalg.norm(d) * rng.uniform(0.5, 1.5))
        pts, ok = [], True
        for _p in range(4):
            for _try in range(100):
                u, v = rng.uniform(0, width), rng.uniform(0, height)
                z = rng.uniform(2, 10)
                Xc = z * np.array([(u - width / 2) / f, (v - height / 2) / f, 1.0])
                proj = []
                good = True
                for k in range(3):
                    xk = Rv[k] @ Xc + Tv[k]
                    if xk[2] <= 0:
                        good = False
                        break
                    uk, vk = f * xk[0] / xk[2] + width / 2, f * xk[1] / xk[2] + height / 2
                    if not (0 <= uk < width and 0 <= vk < height):
                        good = False
                        break
                    proj.append((uk, vk))
                if good:
                    pts.append((Xc, proj))
                    break
            else:
                ok = False
                break
        if ok and abs(Tv[1][2]) > 0.05:
            break

    def pack(pixlists):
        out = []
        for proj in pixlists:
            for (uk, vk) in proj:
                out += [(uk - width / 2) / scale, (vk - height / 2) / scale]
        return np.array(out, dtype=np.complex128)

    clean = [proj for (_, proj) in pts]
    noisy = [[(uk + rng.normal(0, noise_px), vk + rng.normal(0, noise_px)) for (uk, vk) in proj]
             for proj in clean]
    sz = Tv[1][2]
    x = [scale / f] + list(_quat_of(Rv[1])) + list(_quat_of(Rv[2])) + \
        [Tv[1][0] / sz, Tv[1][1] / sz] + list(Tv[2] / sz) + [Xc[2] / sz for (Xc, _) in pts]
    return pack(noisy), dict(p_clean=pack(clean), x_true=np.array(x, dtype=np.complex128), f=f,
                             R=Rv, T=Tv)


def p3p_scene(seed: int, noise_px: float = 0.5, f: float = 1000.0, width: int = 1920,
              height: int = 1080):
    """Synthetic P3P instance: three points with pixels uniform in the image
    and depths U[2, 10] in the camera frame; image points with N(0,
    noise_px) pixel noise, normalised by K^-1; a, b, c from the exact 3D
    points (a P3P solver knows the world points).  Returns (p1, truth) with
    truth['rho'] the true depths (an exact root of the noise-free p_clean)."""
    rng = np.random.default_rng([seed, 0x93])
    Kinv = np.linalg.inv(np.array([[f, 0, width / 2], [0, f, height / 2], [0, 0, 1.0]]))
    pix = [(rng.uniform(0, width), rng.uniform(0, height)) for _ in range(3)]
    depth = rng.uniform(2.0, 10.0, 3)
    G = [d * (Kinv @ np.array([u, v, 1.0])) for d, (u, v) in zip(depth, pix)]
    abc = [float((G[1] - G[0]) @ (G[1] - G[0])), float((G[2] - G[0]) @ (G[2] - G[0])),
           float((G[1] - G[0]) @ (G[2] - G[0]))]

    def pack(pixels):
        out = []
        for (u, v) in pixels:
            g = Kinv @ np.array([u, v, 1.0])
            out += [g[0], g[1]]
        return np.array(out + abc, dtype=np.complex128)
    noisy = [(u + rng.normal(0, noise_px), v + rng.normal(0, noise_px)) for (u, v) in pix]
    return pack(noisy), dict(p_clean=pack(pix), rho=depth.astype(np.complex128))


def pose5_scene(seed: int, noise_px: float = 0.5, f: float = 1000.0, width: int = 1920,
                height: int = 1080, max_angle_deg: float = 30.0):
    """Synthetic two-view scene for pose5_depth_family: camera 1 at the
    identity, camera 2 rotated about a random axis by U[0, max_angle_deg]
    degrees and translated by a random direction x U[0.5, 1.5] (with a
    nonzero third component); five points with pixels uniform in image 1 and
    depth U[2, 10], visible in front of camera 2; N(0, noise_px) pixel noise.
    Returns (p1, truth); truth['x_true'] solves the noise-free p_clean (depths
    and translation scaled by 1 / T_z onto the chart T = (a, b, 1))."""
    rng = np.random.default_rng([seed, 0x5D])
    K = np.array([[f, 0, width / 2], [0, f, height / 2], [0, 0, 1.0]])
    Kinv = np.linalg.inv(K)
    for _attempt in range(1000):
        ax = rng.standard_normal(3)
        R = _rot_axis_angle(ax, np.deg2rad(rng.uniform(0, max_angle_deg)))
        T = rng.standard_normal(3)
        T = T / np.linalg.norm(T) * rng.uniform(0.5, 1.5)
        if abs(T[2]) < 0.2:
            continue
        pts, ok = [], True
        for _ in range(5):
            u, v = rng.uniform(0, width), rng.uniform(0, height)
            d = rng.uniform(2.0, 10.0)
            X1 = d * (Kinv @ np.array([u, v, 1.0]))
            X2 = R @ X1 + T
            if X2[2] <= 0.1:
                ok = False
                break
            h = K @ (X2 / X2[2])
            if not (0 <= h[0] < width and 0 <= h[1] < height):
                ok = False
                break
            pts.append(((u, v), (h[0], h[1]), d, X2[2]))
        if ok:
            break

    def pack(points):
        out = []
        for (u, v), (ub, vb) in points:
            g = Kinv @ np.array([u, v, 1.0])
            gb = Kinv @ np.array([ub, vb, 1.0])
            out += [g[0], g[1], gb[0], gb[1]]
        return np.array(out, dtype=np.complex128)
    clean = [(a, b) for (a, b, _, _) in pts]
    noisy = [((a[0] + rng.normal(0, noise_px), a[1] + rng.normal(0, noise_px)),
              (b[0] + rng.normal(0, noise_px), b[1] + rng.normal(0, noise_px))) for (a, b) in clean]
    sz = T[2]
    x = [d / sz for (_, _, d, _) in pts] + [db / sz for (_, _, _, db) in pts] + \
        list(_quat_of(R)) + [T[0] / sz, T[1] / sz]
    return pack(noisy), dict(p_clean=pack(clean), x_true=np.array(x, dtype=np.complex128), R=R,
                             T=T)


def dense_parameter_family(n: int, d: int, seed: int):
    """A dense random system written as a parameter family whose parameters
    are its coefficients: F(x; p) = sum_k p_k x^alpha_k (one parameter per
    term).  Returns (system, p1, p0) with p1 = the random coefficients and
    p0 = gamma * G embedded in the same support (coefficient gamma on
    x_i^d, -gamma on the constant of equation i, 0 elsewhere), so that
    F(x; (1-t) p0 + t p1) = (1-t) gamma G(x) + t F(x): the total-degree
    homotopy written as a parameter homotopy.
    """
    base = dense_system(n, d, seed)
    T = base.n_terms
    sys_ = TermSystem(n=n, term_eq=base.term_eq, term_coef=np.ones(T, np.complex128),
                      term_exp=base.term_exp, term_param=np.arange(T, dtype=np.int32)[:, None],
                      n_params=T, name=f"dense_param_n{n}_d{d}_s{seed}")
    g = unit_gamma(seed)
    p0 = np.zeros(T, np.complex128)
    for k in range(T):
        i = int(base.term_eq[k])
        e = base.term_exp[k]
        if e.sum() == 0:
            p0[k] = -g
        elif e[i] == d and e.sum() == d:
            p0[k] = g
    return sys_, base.term_coef.copy(), p0


# The dense total-degree sweep: quadratics n = 8, 10, 12 (256 / 1024 / 4096
# paths) and cubics n = 6, 8 (729 / 6561 paths), 16 systems per size, the
# stand-in for the paper's Table 1 benchmark systems at several sizes.
DENSE_SWEEP_SIZES = ((8, 2), (10, 2), (12, 2), (6, 3), (8, 3))
DENSE_SWEEP_SYSTEMS = 16
DENSE_SWEEP_SEED0 = 100


def dense_sweep(rank: int = 0, systems: int = DENSE_SWEEP_SYSTEMS):
    """Per size class: dict(n, d, base, coefs [systems, T], seeds, gamma).

    Replica `rank` gets its own seeds; all systems of a class share the
    class's gamma (the homotopy constant of its first seed)."""
    out = []
    for si, (n, d) in enumerate(DENSE_SWEEP_SIZES):
        seeds = [DENSE_SWEEP_SEED0 + 1000 * rank + 100 * si + k for k in range(systems)]
        base, coefs = dense_batch(n, d, seeds)
        out.append(dict(n=n, d=d, base=base, coefs=coefs, seeds=seeds, gamma=unit_gamma(seeds[0])))
    return out


def total_degree_as_parameter_family(system: TermSystem, gamma: complex):
    """A total-degree homotopy written as a parameter homotopy: the family
    F(x; p) = sum_k p_k x^alpha_k over the union of the monomials of F and of
    the start system G_i = x_i^{d_i} - 1, with p1 = F's coefficients (0 where
    only G has a monomial) and p0 = gamma G's (gamma on x_i^{d_i}, -gamma on
    the constant of equation i, 0 elsewhere), so that F(x; (1-t) p0 + t p1) =
    (1-t) gamma G(x) + t F(x).  Returns (family system, p0, p1, start) with
    start the prod d_i roots of unity, path k from the base-d_i digits of k
    (variable 1 least significant)."""
    n = system.n
    deg = system.degrees()
    terms = {}
    for k in range(system.n_terms):
        key = (int(system.term_eq[k]), tuple(int(e) for e in system.term_exp[k]))
        terms[key] = terms.get(key, 0) + complex(system.term_coef[k])
    g = {}
    for i in range(n):
        e = [0] * n
        e[i] = int(deg[i])
        g[(i, tuple(e))] = complex(gamma)
        g[(i, (0,) * n)] = g.get((i, (0,) * n), 0) - complex(gamma)
    keys = sorted(set(terms) | set(g))
    T = len(keys)
    sys_ = TermSystem(n=n, term_eq=np.array([k[0] for k in keys]), term_coef=np.ones(T),
                      term_exp=np.array([k[1] for k in keys]).reshape(T, n),
                      term_param=np.arange(T, dtype=np.int32)[:, None], n_params=T,
                      name=f"{system.name}_as_parameter_family")
    p0 = np.array([g.get(k, 0) for k in keys], np.complex128)
    p1 = np.array([terms.get(k, 0) for k in keys], np.complex128)
    paths = int(np.prod(deg))
    start = np.zeros((paths, n), np.complex128)
    for p in range(paths):
        r = p
        for i in range(n):
            d = int(deg[i])
            start[p, i] = np.exp(2j * np.pi * (r % d) / d)
            r //= d
    return sys_, p0, p1, start

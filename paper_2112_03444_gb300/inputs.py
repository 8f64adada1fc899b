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
target systems F(x) (Sec. 3, Eq. 1) are sums of such terms; the homogenised
term tuples of Sec. 6 are derived from this list by the library.
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

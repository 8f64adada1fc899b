"""The worked example of Sec. 6 ("Parallel Evaluations of the Jacobian and
Vectors") as test data: the paper's homogenised term tuples of two Jacobian
elements (tests/golden/sec6_term_tuples.json) and a two-variable parameter
family whose Jacobian has exactly those elements:

    F1 = a1 x1^2 + 2 a2 x1^2 x2 + 8 a3 x1 x2^2   dF1/dx1 = A = 2 a1 x1 + 4 a2 x1 x2 + 8 a3 x2^2
    F2 = 5/2 a4 x1^2 x2 + 7 a5 x1 x2^2           dF2/dx1 = B = 5 a4 x1 x2 + 7 a5 x2^2

with the coefficients a = (a1 .. a5) as the family's parameters, so that
along the homotopy a(t) = (1 - t) a(0) + t a(1) as the paper describes
("the coefficients a_i are linear interpolation of corresponding elements in
the start and target systems")."""
import json
import os

import numpy as np

from paper_2112_03444_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def tuples():
    with open(os.path.join(HERE, "golden", "sec6_term_tuples.json")) as f:
        return json.load(f)


def tuple_value(tup, a, x):
    """U = sum_k s_k a_{j_k} x_{m1} x_{m2} with the auxiliary x3 = 1
    (indices 1-based as printed)."""
    X = [x[0], x[1], 1.0]
    return sum(s * a[j - 1] * X[m1 - 1] * X[m2 - 1] for s, j, m1, m2 in tup)


def family():
    # (equation, coefficient, exponents of x1 and x2, parameter index)
    terms = [(0, 1.0, (2, 0), 0), (0, 2.0, (2, 1), 1), (0, 8.0, (1, 2), 2),
             (1, 2.5, (2, 1), 3), (1, 7.0, (1, 2), 4)]
    return inputs.TermSystem(
        n=2, term_eq=np.array([e for e, _, _, _ in terms]),
        term_coef=np.array([c for _, c, _, _ in terms], np.complex128),
        term_exp=np.array([x for _, _, x, _ in terms]),
        term_param=np.array([[p] for _, _, _, p in terms]), n_params=5, name="sec6_example")


def parameters(seed=0):
    rng = np.random.default_rng(seed)
    p0 = rng.normal(size=5) + 1j * rng.normal(size=5)
    p1 = rng.normal(size=5) + 1j * rng.normal(size=5)
    return p0, p1

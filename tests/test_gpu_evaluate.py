"""The device evaluator (row a3: H, dH/dx and dH/dt in one pass, Sec. 6)
called through hc_evaluate, point by point against the FP64 oracle's
evaluation, in each arithmetic (FP64, double-float, FP32), for dense
total-degree systems, parameter families and coefficient interpolation;
and the Jacobian of the Sec. 6 worked example against the paper's printed
term tuples."""
import os

import numpy as np
import pytest

import oracle
from oracle import KIND_COEFFICIENT, KIND_PARAMETER, OracleProblem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STARTS = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")
# relative tolerance per arithmetic, against the scale of the largest entry
TOL = {0: 1e-13, 2: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc as mod
    return mod


def _close(got, want, tol):
    scale = max(1.0, float(np.max(np.abs(want))))
    err = float(np.max(np.abs(got - want)))
    assert err <= tol * scale, (err, scale)


def _points(n, k, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    x = scale * (rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n)))
    t = rng.uniform(size=k)
    t[0], t[-1] = 0.0, 1.0
    return x, t


@pytest.mark.parametrize("precision", [0, 2, 1], ids=["fp64", "df", "fp32"])
@pytest.mark.parametrize("n,d", [(1, 2), (3, 2), (6, 2), (9, 2), (12, 2), (2, 3), (5, 3), (8, 3)])
def test_dense_evaluation_matches_oracle(hc, n, d, precision):
    from paper_2112_03444_gb300 import inputs
    seeds = [300 + n, 310 + n]
    base, coefs = inputs.dense_batch(n, d, seeds)
    gamma = inputs.unit_gamma(seeds[0])
    pr = hc.Problem(base, gamma=gamma)
    x, t = _points(n, 40, n * 10 + d)
    inst = np.arange(40) % 2
    H, Hx, Ht = pr.evaluate(x, t, instance=inst, coef=coefs, precision=precision)
    for k in range(40):
        ref = oracle.OracleProblem(base, gamma=gamma, coef=coefs[inst[k]]).eval(x[k], t[k])
        _close(H[k], ref[0], TOL[precision])
        _close(Hx[k], ref[1], TOL[precision])
        _close(Ht[k], ref[2], TOL[precision])


@pytest.mark.parametrize("precision", [0, 2, 1], ids=["fp64", "df", "fp32"])
@pytest.mark.parametrize("name,kind", [("triangulation4", KIND_PARAMETER),
                                       ("p3p", KIND_PARAMETER),
                                       ("p3p", KIND_COEFFICIENT),
                                       ("trifocal_f", KIND_PARAMETER)])
def test_family_evaluation_matches_oracle(hc, name, kind, precision):
    from paper_2112_03444_gb300 import inputs
    fam = {"triangulation4": lambda: inputs.triangulation_family(4),
           "p3p": inputs.p3p_family, "trifocal_f": inputs.trifocal_family}[name]()
    z = np.load(os.path.join(STARTS, f"{name}.npz"))
    rng = np.random.default_rng(11)
    P = len(z["p0"])
    p1 = rng.normal(size=(3, P)) + 1j * rng.normal(size=(3, P))
    hk = hc.HC_PARAMETER if kind == KIND_PARAMETER else hc.HC_COEFFICIENT
    pr = hc.Problem(fam.system, kind=hk, p0=z["p0"], start=z["start"][:4])
    S = len(z["start"])
    x = z["start"][np.arange(24) % S] + 0.1 * (rng.normal(size=(24, fam.system.n)) +
                                                1j * rng.normal(size=(24, fam.system.n)))
    t = rng.uniform(size=24)
    inst = np.arange(24) % 3
    H, Hx, Ht = pr.evaluate(x, t, instance=inst, p1=p1, precision=precision)
    for k in range(24):
        ref = OracleProblem(fam.system, kind=kind, p0=z["p0"], p1=p1[inst[k]]).eval(x[k], t[k])
        _close(H[k], ref[0], TOL[precision])
        _close(Hx[k], ref[1], TOL[precision])
        _close(Ht[k], ref[2], TOL[precision])


@pytest.mark.parametrize("precision", [0, 2, 1], ids=["fp64", "df", "fp32"])
def test_jacobian_matches_the_paper_term_tuples(hc, precision):
    """Sec. 6: dH/dx (1,1) and (2,1) of the example family equal the paper's
    tuples for A and B at a(t) = (1 - t) a(0) + t a(1), x3 = 1."""
    import sec6_example as ex
    tup = ex.tuples()
    fam = ex.family()
    p0, p1 = ex.parameters(2)
    pr = hc.Problem(fam, kind=hc.HC_PARAMETER, p0=p0, start=np.ones((1, 2)))
    x, t = _points(2, 16, 5)
    _, Hx, _ = pr.evaluate(x, t, p1=p1[None, :], precision=precision)
    for k in range(16):
        a = (1 - t[k]) * p0 + t[k] * p1
        A = ex.tuple_value(tup["A"], a, x[k])
        B = ex.tuple_value(tup["B"], a, x[k])
        assert abs(Hx[k, 0, 0] - A) <= TOL[precision] * max(1, abs(A)), (k, Hx[k, 0, 0], A)
        assert abs(Hx[k, 1, 0] - B) <= TOL[precision] * max(1, abs(B)), (k, Hx[k, 1, 0], B)


def test_evaluate_rejects_bad_instance(hc):
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(2, 2, [1])
    pr = hc.Problem(base)
    with pytest.raises(hc.HCError):
        pr.evaluate(np.zeros((1, 2)), [0.5], instance=[3], coef=coefs)


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "df"])
def test_dense_evaluation_far_from_the_origin(hc, precision):
    """Points of norm ~1e3 (a diverging path's range): the double-float
    evaluation keeps its relative accuracy (FP32 exponent range suffices)."""
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(6, 3, [77])
    gamma = inputs.unit_gamma(77)
    pr = hc.Problem(base, gamma=gamma)
    x, t = _points(6, 12, 9, scale=1e3)
    H, Hx, Ht = pr.evaluate(x, t, coef=coefs, precision=precision)
    op = oracle.OracleProblem(base, gamma=gamma, coef=coefs[0])
    for k in range(12):
        ref = op.eval(x[k], t[k])
        _close(H[k], ref[0], TOL[precision])
        _close(Hx[k], ref[1], TOL[precision])
        _close(Ht[k], ref[2], TOL[precision])

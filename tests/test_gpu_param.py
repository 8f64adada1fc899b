"""GPU parity of the parameter-homotopy (term-tuple) tracker against the
FP64 oracle on the same seeded inputs: status counts per class equal and
endpoints matched bijectively within 1e-8 relative."""
import os

import numpy as np
import pytest

import oracle
from oracle import KIND_PARAMETER, OracleProblem
from hcmatch import distinct, match, rel_dist, same_set

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STARTS = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")
TOL = 1e-8


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc as mod
    return mod


# Benign changes of the tracker settings: a path whose oracle classification
# changes under one of them is ill-determined (it passes so close to a
# singularity that the rounding of any FP64 evaluation order decides it).
PERTURB = [dict(newton_tol=5e-9), dict(newton_tol=2e-8), dict(dt_init=0.005), dict(dt_init=0.02)]


def _ill_determined(ref_problem, start_row, base_class):
    for s in PERTURB:
        r = ref_problem.track(start=start_row[None, :], settings=s)
        if (r["status"][0] & 0x7F) != base_class:
            return True
    return False


def _check(hc, system, p0, p1s, start, precision, symmetries=(), kind=None):
    """Exact status counts and bijective endpoint match, on every path whose
    oracle outcome is stable; a path on which the GPU and the oracle differ
    must be ill-determined (see PERTURB), at most 1 % of an instance, and a
    finite GPU endpoint there must still pass the backward-error test."""
    kind = hc.HC_PARAMETER if kind is None else kind
    pr = hc.Problem(system, kind=kind, p0=p0, start=start,
                    settings=dict(precision=precision), symmetries=symmetries)
    b = pr.track(n_instances=len(p1s), p1=np.array(p1s)).wait()
    for s, p1 in enumerate(p1s):
        refp = OracleProblem(system, kind=int(kind), p0=p0, p1=p1)
        ref = refp.track(start=start)
        gc, oc = b.status[s] & 0x7F, ref["status"] & 0x7F
        keep = np.ones(len(start), bool)
        for i in np.nonzero(gc != oc)[0]:
            assert _ill_determined(refp, start[i], oc[i]), (s, int(i), int(gc[i]), int(oc[i]))
            if gc[i] == oracle.FINITE:
                assert b.be[s][i] <= 1e-10, (s, int(i), float(b.be[s][i]))
            keep[i] = False
        assert (~keep).sum() <= max(1, len(start) // 100), (s, int((~keep).sum()))
        got = oracle.status_counts(b.status[s][keep])
        want = oracle.status_counts(ref["status"][keep])
        assert got == want, (s, got, want)
        fg = keep & (gc == oracle.FINITE)
        fo = keep & (oc == oracle.FINITE)
        ok, msg = same_set(b.x[s][fg], ref["x"][fo], TOL)
        assert ok, (s, msg)
    return b


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
@pytest.mark.parametrize("n,d,seed", [(1, 3, 71), (3, 2, 72), (4, 2, 73), (2, 3, 74), (5, 2, 75)])
def test_dense_parameter_family_matches_oracle(hc, n, d, seed, precision):
    from paper_2112_03444_gb300 import inputs
    sys_, p1, p0 = inputs.dense_parameter_family(n, d, seed)
    base = OracleProblem(inputs.dense_system(n, d, seed))
    start = np.array([base.start_point(k) for k in range(d ** n)])
    p1b = p1 * np.exp(0.3j)  # a second instance: rotated coefficients
    _check(hc, sys_, p0, [p1, p1b], start, precision)


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
def test_triangulation_matches_oracle(hc, precision):
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1s = [inputs.triangulation_scene(s)[0] for s in (31, 32)]
    _check(hc, fam.system, z["p0"], p1s, z["start"], precision)


def _family(name):
    from paper_2112_03444_gb300 import inputs
    return {"p3p": (inputs.p3p_family(), inputs.p3p_scene),
            "triangulation2": (inputs.triangulation_family(2),
                               lambda s: inputs.triangulation_scene(s, views=2)),
            "pose5_depth": (inputs.pose5_depth_family(), inputs.pose5_scene)}[name]


@pytest.mark.parametrize("sym", [False, True], ids=["all_starts", "orbit_reps"])
@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
@pytest.mark.parametrize("name", ["p3p", "triangulation2", "pose5_depth"])
def test_more_vision_problems_match_oracle(hc, name, precision, sym):
    """The other formulations of Sec. 4: P3P in the depths (3 x 3), two-view
    triangulation (5 x 5) and relative pose with depths (16 x 16), each from
    its oracle monodromy start set to three noisy scenes."""
    fam, scene = _family(name)
    if sym and not fam.sign_masks:
        pytest.skip("no sign symmetry")
    z = np.load(os.path.join(STARTS, f"{name}.npz"))
    p1s = [scene(s)[0] for s in (61, 62, 63)]
    _check(hc, fam.system, z["p0"], p1s, z["start"], precision,
           symmetries=fam.sign_masks if sym else ())


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
@pytest.mark.parametrize("name", ["triangulation4", "p3p", "pose5_depth"])
def test_coefficient_interpolation_matches_oracle(hc, name, precision):
    """The coefficient-interpolation homotopy of Sec. 6 (HC_COEFFICIENT: the
    term coefficients, products of parameters, interpolated linearly) against
    the oracle's own coefficient-interpolation mode, from the monodromy start
    sets to three noisy scenes."""
    from paper_2112_03444_gb300 import inputs
    if name == "triangulation4":
        fam, scene = inputs.triangulation_family(4), inputs.triangulation_scene
    else:
        fam, scene = _family(name)
    z = np.load(os.path.join(STARTS, f"{name}.npz"))
    p1s = [scene(s)[0] for s in (71, 72, 73)]
    _check(hc, fam.system, z["p0"], p1s, z["start"], precision, kind=hc.HC_COEFFICIENT)


def test_parameter_batch_device_pointers(hc):
    import torch
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1s = np.array([inputs.triangulation_scene(s)[0] for s in (41, 42, 43)])
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"])
    hb = pr.track(n_instances=3, p1=p1s).wait()
    dev = torch.device("cuda")
    P, n = pr.paths, 14
    xo = torch.zeros((3, P, n), dtype=torch.complex128, device=dev)
    so = torch.zeros((3, P), dtype=torch.uint8, device=dev)
    to = torch.zeros((3, P, 3), dtype=torch.int32, device=dev)
    db = pr.track(n_instances=3, p1=torch.from_numpy(p1s).to(dev), device=True, x_out=xo,
                  status_out=so, steps_out=to, stream=torch.cuda.current_stream().cuda_stream).wait()
    assert np.array_equal(so.cpu().numpy(), hb.status)
    assert np.array_equal(xo.cpu().numpy(), hb.x)


def test_trifocal_sampled_starts_match_oracle(hc):
    """Trifocal pose with unknown focal length, 192 sampled start roots and
    two noisy scenes: the plain FP64 kernel and the oracle on the same starts,
    path by path (nothing is re-tracked, so a sample is a fair test)."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    sel = np.random.default_rng(7).choice(len(z["start"]), size=192, replace=False)
    p1s = [inputs.trifocal_scene(s)[0] for s in (51, 52)]
    _check(hc, fam.system, z["p0"], p1s, z["start"][sel], 0)


def test_trifocal_full_start_set_recovers_true_pose(hc):
    """All 5344 start roots to a noise-free scene on the GPU (mixed
    precision, orbit representatives): the true pose is an endpoint."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    _, truth = inputs.trifocal_scene(3, noise_px=0.0)
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"],
                    symmetries=fam.sign_masks)
    b = pr.track(n_instances=1, p1=truth["p_clean"][None, :]).wait()
    fin = b.x[0][(b.status[0] & 0x7F) == hc.PATH_FINITE]
    xt = truth["x_true"]
    best = np.inf
    for s12 in (1, -1):
        for s13 in (1, -1):
            v = xt.copy()
            v[1:5] *= s12
            v[5:9] *= s13
            best = min(best, float(np.min(np.max(np.abs(fin - v), axis=1))))
    assert best < 1e-8, best


def _trifocal_golden():
    return np.load(os.path.join(ROOT, "tests", "golden", "trifocal_oracle.npz"))


@pytest.mark.parametrize("sym", [False, True], ids=["all_starts", "orbit_reps"])
def test_trifocal_full_start_set_matches_oracle_golden(hc, sym):
    """All 5344 start roots, two noisy scenes, mixed precision (duplicate
    detection and re-tracking over the full set), against the oracle's
    stored outcome on every path (tests/golden/trifocal_oracle.npz): status
    counts equal and every finite GPU endpoint matched one to one to an
    oracle endpoint within 1e-8 relative (through the golden's random linear
    projection of the endpoints), on every path whose oracle outcome is
    stable; a path on which the two differ must be ill-determined (PERTURB),
    at most 1 % of the starts."""
    from scipy.spatial import cKDTree
    from paper_2112_03444_gb300 import inputs
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    gold = _trifocal_golden()
    c = gold["proj_coef"]
    p1 = np.stack([inputs.trifocal_scene(int(sd))[0] for sd in gold["scenes"]])
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"],
                    symmetries=fam.sign_masks if sym else ())
    b = pr.track(n_instances=len(p1), p1=p1).wait()
    for k in range(len(p1)):
        ost = gold[f"status{k}"] & 0x7F
        gst = b.status[k] & 0x7F
        keep = np.ones(len(ost), bool)
        differ = np.nonzero(gst != ost)[0]
        assert len(differ) <= len(ost) // 100, (k, len(differ))
        refp = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=z["p0"], p1=p1[k])
        for i in differ:
            assert _ill_determined(refp, z["start"][i], ost[i]), (k, int(i), int(gst[i]),
                                                                   int(ost[i]))
            if gst[i] == oracle.FINITE:
                assert b.be[k][i] <= 1e-10, (k, int(i))
            keep[i] = False
        assert oracle.status_counts(b.status[k][keep]) == \
            oracle.status_counts(gold[f"status{k}"][keep])
        fg = keep & (gst == oracle.FINITE)
        fo = keep & (ost == oracle.FINITE)
        gp = b.x[k][fg] @ c
        op = gold[f"proj{k}"][fo]
        tol = np.sum(np.abs(c)) * TOL * np.maximum(1.0, gold[f"xnorm{k}"][fo])
        tree = cKDTree(np.stack([op.real, op.imag], axis=1))
        d, idx = tree.query(np.stack([gp.real, gp.imag], axis=1), k=1)
        assert np.all(d <= tol[idx]), (k, float(np.max(d / tol[idx])))
        assert len(np.unique(idx)) == len(idx), k          # one to one
        assert distinct(b.x[k][gst == oracle.FINITE]) == int((gst == oracle.FINITE).sum())


def test_trifocal_orbit_reduction_is_exact(hc):
    """Tracking one start per orbit of the two quaternion sign symmetries and
    writing the signed images gives bit for bit what tracking every start
    gives (plain FP64, where nothing is re-tracked): the homotopy is
    equivariant and the evaluation and the solve treat negated columns
    alike in floating point."""
    from scipy.spatial import cKDTree
    from paper_2112_03444_gb300 import inputs
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    S = z["start"]
    # The committed set is symmetric to rounding only (monodromy found each
    # sign image by tracking): make it exactly so, every start the exact
    # sign image of the lowest-index member of its orbit.
    signs = []
    for e in range(4):
        m = sum(fam.sign_masks[k] for k in range(2) if e >> k & 1)
        signs.append(np.array([-1.0 if m >> j & 1 else 1.0 for j in range(18)]))
    tree = cKDTree(np.concatenate([S.real, S.imag], 1))
    exact = S.copy()
    for j in range(len(S)):
        best, sg = j, signs[0]
        for e in range(1, 4):
            y = signs[e] * S[j]
            d, i = tree.query(np.concatenate([y.real, y.imag]), p=np.inf)
            assert d <= 1e-9 * max(1.0, float(np.max(np.abs(y))))   # the library's rule
            if i < best:
                best, sg = i, signs[e]
        exact[j] = sg * S[best]
    p1 = inputs.trifocal_scene(55)[0][None, :]
    out = []
    for sym in ((), fam.sign_masks):
        pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=exact,
                        settings=dict(precision=0), symmetries=sym)
        out.append(pr.track(n_instances=1, p1=p1).wait())
    assert np.array_equal(out[0].status, out[1].status)
    assert np.array_equal(out[0].x, out[1].x, equal_nan=True)   # failed paths may hold NaN
    assert np.array_equal(out[0].steps, out[1].steps)
    # the reduced batch tracked a quarter of the paths
    assert out[1].result["steps_accepted"] * 4 == out[0].result["steps_accepted"]


def test_symmetry_validation(hc):
    """A mask under which some term has odd degree, or a start set that is not
    closed under the masks, is refused at creation."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    with pytest.raises(hc.HCError) as e:
        hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"],
                   symmetries=[1 << 9])          # the translation unknown a
    assert e.value.code == hc.HC_ERR_INVALID
    with pytest.raises(hc.HCError) as e:
        hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"][:5],
                   symmetries=fam.sign_masks)
    assert e.value.code == hc.HC_ERR_INVALID


def _poly(n, polys):
    from paper_2112_03444_gb300 import inputs
    return inputs.system_from_polys(n, polys)


EDGE_CASES = {
    # x_i^2 = a_i, a_i > 0: 8 real roots
    "decoupled_real_squares": (3, [{(2, 0, 0): 1, (0, 0, 0): -2.0}, {(0, 2, 0): 1, (0, 0, 0): -0.5},
                                   {(0, 0, 2): 1, (0, 0, 0): -3.0}], 5),
    # x^2 = 1 + i: two finite non-real roots
    "complex_square": (1, [{(2,): 1, (0,): -(1 + 1j)}], 6),
    # x1^2 = a, x2^2 = x1 + b
    "triangular": (2, [{(2, 0): 1, (0, 0): -(1.5 - 0.5j)},
                       {(0, 2): 1, (1, 0): -1, (0, 0): -(0.25 + 2j)}], 8),
    # x1 x2 = 1, x1 x2 + x1 = 2: one finite root, three paths to infinity
    "deficient": (2, [{(1, 1): 1, (0, 0): -1}, {(1, 1): 1, (1, 0): 1, (0, 0): -2}], 9),
    # x^2 = 0: both paths end at a double root
    "double_root": (1, [{(2,): 1.0}], 10),
}


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
@pytest.mark.parametrize("case", sorted(EDGE_CASES))
def test_edge_cases_match_oracle_exactly(hc, case, precision):
    """The method's degenerate cases (paths to infinity, a double root, real
    roots), each a total-degree homotopy written as a parameter family: the
    GPU's statuses equal the oracle's path by path -- diverged, singular,
    failed and the real bit included -- and the finite endpoints match."""
    from paper_2112_03444_gb300 import inputs
    n, polys, gseed = EDGE_CASES[case]
    fam, p0, p1, start = inputs.total_degree_as_parameter_family(_poly(n, polys),
                                                                 inputs.unit_gamma(gseed))
    pr = hc.Problem(fam, kind=hc.HC_PARAMETER, p0=p0, start=start,
                    settings=dict(precision=precision))
    b = pr.track(n_instances=1, p1=p1[None, :]).wait()
    ref = OracleProblem(fam, kind=KIND_PARAMETER, p0=p0, p1=p1).track(start=start)
    assert np.array_equal(b.status[0], ref["status"]), (b.status[0], ref["status"])
    fin = (ref["status"] & 0x7F) == oracle.FINITE
    ok, msg = same_set(b.x[0][fin], ref["x"][fin], TOL)
    assert ok, msg
    # and the oracle's parameter form is its total-degree homotopy (pinned there)
    td = OracleProblem(_poly(n, polys), gamma=inputs.unit_gamma(gseed)).track()
    assert oracle.status_counts(td["status"]) == oracle.status_counts(ref["status"])


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
def test_path_to_infinity_is_diverged_like_the_oracle(hc, precision):
    """F(x; p) = (p x - y, p y - 1) has the single root y = 1/p, x = 1/p^2;
    from p = 1 to p = 0 the path leaves every bounded set like (1-t)^-2 and
    passes the divergence radius before the step size underflows: both the
    GPU and the oracle classify it HC_PATH_DIVERGED (the oracle's class is
    checked too, so the test fails if either changes)."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.TermSystem(n=2, term_eq=[0, 0, 1, 1], term_coef=[1, -1, 1, -1],
                            term_exp=[[1, 0], [0, 1], [0, 1], [0, 0]],
                            term_param=[[0], [-1], [0], [-1]], n_params=1)
    p0, p1 = np.array([1.0 + 0j]), np.array([0.0 + 0j])
    start = np.array([[1.0, 1.0]], np.complex128)
    pr = hc.Problem(fam, kind=hc.HC_PARAMETER, p0=p0, start=start,
                    settings=dict(precision=precision))
    b = pr.track(n_instances=1, p1=p1[None, :]).wait()
    ref = OracleProblem(fam, kind=KIND_PARAMETER, p0=p0, p1=p1).track(start=start)
    assert ref["status"][0] == oracle.DIVERGED
    assert b.status[0][0] == ref["status"][0]


ENDGAME_CASES = {
    "triple_root": (2, [{(3, 0): 1.0, (2, 0): -3.0, (1, 0): 3.0, (0, 0): -1.0},
                        {(0, 1): 1.0, (0, 0): -1.0}], 4),
    "double_root": (2, [{(2, 0): 1.0, (1, 0): -2.0, (0, 0): 1.0}, {(0, 1): 1.0, (0, 0): -1.0}], 3),
    "deficient": EDGE_CASES["deficient"],
    "decoupled_real_squares": EDGE_CASES["decoupled_real_squares"],
}


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
@pytest.mark.parametrize("case", sorted(ENDGAME_CASES))
def test_endgame_matches_oracle(hc, case, precision):
    """The power-series endgame (settings.endgame = 1) against the oracle's
    own endgame: statuses path by path (singular endpoints of multiple roots
    included) and the finite and singular endpoints within 1e-8.  In mixed
    precision the endgame runs in the last re-tracking tier (double-float
    arithmetic by default), which gets the paths that fail near their end."""
    from paper_2112_03444_gb300 import inputs
    n, polys, gseed = ENDGAME_CASES[case]
    fam, p0, p1, start = inputs.total_degree_as_parameter_family(_poly(n, polys),
                                                                 inputs.unit_gamma(gseed))
    pr = hc.Problem(fam, kind=hc.HC_PARAMETER, p0=p0, start=start,
                    settings=dict(precision=precision, endgame=1))
    b = pr.track(n_instances=1, p1=p1[None, :]).wait()
    ref = OracleProblem(fam, kind=KIND_PARAMETER, p0=p0, p1=p1).track(
        start=start, settings=dict(endgame=1))
    assert np.array_equal(b.status[0] & 0x7F, ref["status"] & 0x7F), (b.status[0], ref["status"])
    for cls in (oracle.FINITE, oracle.SINGULAR):
        m = (ref["status"] & 0x7F) == cls
        if m.any():
            assert np.max(rel_dist(b.x[0][m], ref["x"][m])) <= TOL, cls

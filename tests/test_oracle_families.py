"""Pins of the parameter-homotopy workloads and of the oracle's monodromy
start sets (CPU only)."""
import os

import numpy as np
import pytest

import oracle
from oracle import KIND_PARAMETER, OracleProblem, monodromy
from paper_2112_03444_gb300 import inputs
from hcmatch import same_set, distinct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STARTS = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")


def test_dense_parameter_family_equals_total_degree_homotopy():
    """F(x; (1-t) p0 + t p1) with p0 = gamma*G is the total-degree homotopy:
    the parameter-homotopy oracle ends on the same root set as the
    total-degree oracle (itself pinned by Bezout counts and closed forms)."""
    sys_, p1, p0 = inputs.dense_parameter_family(3, 2, 61)
    td = OracleProblem(inputs.dense_system(3, 2, 61), gamma=inputs.unit_gamma(61)).track()
    start = np.array([td_start for td_start in
                      (OracleProblem(inputs.dense_system(3, 2, 61)).start_point(k) for k in range(8))])
    pr = OracleProblem(sys_, kind=KIND_PARAMETER, p0=p0, p1=p1).track(start=start)
    assert oracle.status_counts(pr["status"]) == oracle.status_counts(td["status"])
    ok, msg = same_set(pr["x"], td["x"], 1e-10)
    assert ok, msg


def test_triangulation_formulation_exact_root_on_consistent_data():
    """Noise-free points and consistent essential matrices: the zero correction
    with zero multipliers satisfies every equation (Lagrangian of Sec. 4)."""
    fam = inputs.triangulation_family(4)
    _, truth = inputs.triangulation_scene(11, noise_px=0.0, pose_noise_deg=0.0, pose_noise_t=0.0)
    r = monodromy.residual(fam.system, np.zeros(14), truth["p_clean"])
    assert np.max(np.abs(r)) < 1e-12


def test_triangulation_unknown_and_equation_counts():
    """(N^2 + 3N) / 2 unknowns and equations: 5, 9, 14 for 2, 3, 4 views (Sec. 4)."""
    for N, want in ((2, 5), (3, 9), (4, 14)):
        fam = inputs.triangulation_family(N)
        assert fam.system.n == want == len(fam.unknowns)
        assert fam.system.n_params == 2 * N + 9 * N * (N - 1) // 2
        assert np.all(fam.system.degrees() == 2)


def test_trifocal_formulation_true_pose_is_a_root():
    """Noise-free scene: the true focal length, rotations (as unit quaternions),
    translations in the T12 = (a, b, 1) chart and depths satisfy all 18
    equations; 18 unknowns, 16 point equations + 2 quaternion norms (Sec. 4)."""
    fam = inputs.trifocal_family()
    assert fam.system.n == 18 and len(fam.unknowns) == 18
    for seed in (1, 2, 3):
        _, truth = inputs.trifocal_scene(seed, noise_px=0.0)
        r = monodromy.residual(fam.system, truth["x_true"], truth["p_clean"])
        assert np.max(np.abs(r)) < 1e-10, seed
        # the quaternion sign is a symmetry: -q gives the same rotation
        x2 = truth["x_true"].copy()
        x2[1:5] *= -1
        assert np.max(np.abs(monodromy.residual(fam.system, x2, truth["p_clean"]))) < 1e-10


def test_monodromy_seed_pair_is_a_root():
    for fam in (inputs.triangulation_family(4), inputs.trifocal_family()):
        x0, p0 = monodromy.seed_pair(fam, np.random.default_rng(5))
        assert np.max(np.abs(monodromy.residual(fam.system, x0, p0))) < 1e-9


def test_triangulation_start_set_matches_paper_count():
    """The committed monodromy start set has 296 distinct roots at p0, the
    number of solutions the paper reports for 4-view triangulation (Table 2)."""
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    S, p0 = z["start"], z["p0"]
    assert S.shape == (296, 14)
    assert distinct(S, 1e-6) == 296
    fam = inputs.triangulation_family(4)
    for x in S[::7]:
        r = monodromy.residual(fam.system, x, p0)
        assert np.max(np.abs(r)) < 1e-8


def test_two_view_zero_correction_is_an_endpoint():
    """Two views, noise-free points, consistent E: the zero correction is a
    nonsingular root (one constraint, no redundancy) and the parameter
    homotopy from a monodromy start set must end on it."""
    fam = inputs.triangulation_family(2)
    S, p0, _ = monodromy.solve(fam, seed=1)
    _, truth = inputs.triangulation_scene(4, views=2, noise_px=0.0, pose_noise_deg=0.0,
                                          pose_noise_t=0.0)
    r = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=p0, p1=truth["p_clean"]).track(start=S)
    fin = (r["status"] & 0x7F) == oracle.FINITE
    assert np.any(fin)
    assert np.min(np.max(np.abs(r["x"][fin]), axis=1)) < 1e-12


def test_triangulation_endpoints_are_roots_of_the_target():
    """Track the 296 start roots to a noisy four-view scene: every finite
    endpoint satisfies F(x; p1) = 0 to rounding (checked by evaluation)."""
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1, _ = inputs.triangulation_scene(21)
    r = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=z["p0"], p1=p1).track(start=z["start"])
    fin = (r["status"] & 0x7F) == oracle.FINITE
    assert fin.sum() >= 280
    for x in r["x"][fin][::9]:
        res = monodromy.residual(fam.system, x, p1)
        assert np.max(np.abs(res)) <= 1e-9 * max(1.0, np.max(np.abs(x)) ** 2)


def test_trifocal_start_set_is_closed_under_quaternion_signs():
    """q and -q give the same rotation, so the root set at p0 must be closed
    under flipping either quaternion: 5344 roots = 4 x 1336 poses.  (The
    paper reports 1784 roots for its formulation; this count is recorded.)"""
    from hcmatch import match
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    S, p0 = z["start"], z["p0"]
    assert S.shape == (5344, 18)
    assert distinct(S, 1e-6) == 5344
    for flip in ([1, 2, 3, 4], [5, 6, 7, 8]):
        S2 = S.copy()
        S2[:, flip] *= -1
        idx, d = match(S2, S, 1e-8)
        assert np.max(d) < 1e-8 and len(np.unique(idx)) == len(S)
    fam = inputs.trifocal_family()
    for x in S[::97]:
        assert np.max(np.abs(monodromy.residual(fam.system, x, p0))) < 1e-10


def test_trifocal_tracking_recovers_the_true_pose():
    """Noise-free three-view scene: tracking all start roots from p0 to the
    scene's parameters ends on the true focal length, rotations, translations
    and depths (in one of the four quaternion-sign variants)."""
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(STARTS, "trifocal_f.npz"))
    _, truth = inputs.trifocal_scene(3, noise_px=0.0)
    r = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=z["p0"], p1=truth["p_clean"]).track(
        start=z["start"])
    fin = r["x"][(r["status"] & 0x7F) == oracle.FINITE]
    xt = truth["x_true"]
    best = np.inf
    for s12 in (1, -1):
        for s13 in (1, -1):
            v = xt.copy()
            v[1:5] *= s12
            v[5:9] *= s13
            best = min(best, float(np.min(np.max(np.abs(fin - v), axis=1))))
    assert best < 1e-8, best


# ---------------------------------------------------------------- P3P, 5-point pose + depth
def _closed_under(S, mask, tol=1e-10):
    sg = np.array([-1.0 if mask >> j & 1 else 1.0 for j in range(S.shape[1])])
    for x in S:
        d = np.max(np.abs(S - sg * x), axis=1) / max(1.0, float(np.max(np.abs(x))))
        if np.min(d) > tol:
            return False
    return True


def test_p3p_formulation_and_start_set():
    """P3P in the depths (Sec. 4, Eq. P3PafterElim): the true depths of a
    noise-free scene satisfy the three quadratics; the oracle's monodromy
    start set has the paper's 8 solutions (Table 2), pairwise distinct, each
    a root at p0, closed under rho -> -rho."""
    fam = inputs.p3p_family()
    assert fam.system.n == 3 and np.all(fam.system.degrees() == 2)
    _, truth = inputs.p3p_scene(4, noise_px=0.0)
    assert np.max(np.abs(monodromy.residual(fam.system, truth["rho"], truth["p_clean"]))) < 1e-10
    z = np.load(os.path.join(STARTS, "p3p.npz"))
    S = z["start"]
    assert len(S) == 8 and distinct(S, 1e-6) == 8
    for x in S:
        assert np.max(np.abs(monodromy.residual(fam.system, x, z["p0"]))) < 1e-10
    assert _closed_under(S, 0b111)


def test_p3p_tracking_recovers_true_depths():
    """From the 8 start solutions to a noise-free scene the oracle's parameter
    homotopy ends at the true depths (and their negatives)."""
    fam = inputs.p3p_family()
    z = np.load(os.path.join(STARTS, "p3p.npz"))
    for seed in (5, 6):
        _, truth = inputs.p3p_scene(seed, noise_px=0.0)
        r = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=z["p0"],
                          p1=truth["p_clean"]).track(start=z["start"])
        fin = r["x"][(r["status"] & 0x7F) == oracle.FINITE]
        for sg in (1, -1):
            d = np.max(np.abs(fin - sg * truth["rho"]), axis=1) / np.max(np.abs(truth["rho"]))
            assert np.min(d) < 1e-9, (seed, sg)


def test_pose5_depth_formulation_and_start_set():
    """Relative pose + depth from five points (Sec. 4, Eq. FullRigidMotion):
    16 equations in 16 unknowns; the true pose of a noise-free scene (depths
    and translation on the T = (a, b, 1) chart, unit quaternion) is a root,
    with either quaternion sign; the oracle's monodromy start set is closed
    under q -> -q.  (Our chart formulation has 40 solutions: 10 essential
    matrices, the twisted pair, the quaternion sign; the paper's Table 2
    count of 160 is for its own formulation, whose equations it does not
    print.)"""
    fam = inputs.pose5_depth_family()
    assert fam.system.n == 16 and len(fam.unknowns) == 16 and fam.system.n_params == 20
    for seed in (1, 2):
        _, truth = inputs.pose5_scene(seed, noise_px=0.0)
        x = truth["x_true"]
        assert np.max(np.abs(monodromy.residual(fam.system, x, truth["p_clean"]))) < 1e-10
        x2 = x.copy()
        x2[10:14] *= -1
        assert np.max(np.abs(monodromy.residual(fam.system, x2, truth["p_clean"]))) < 1e-10
    z = np.load(os.path.join(STARTS, "pose5_depth.npz"))
    S = z["start"]
    assert len(S) == 40 and distinct(S, 1e-6) == 40
    assert _closed_under(S, 0b1111 << 10)


def test_pose5_depth_tracking_recovers_true_pose():
    fam = inputs.pose5_depth_family()
    z = np.load(os.path.join(STARTS, "pose5_depth.npz"))
    _, truth = inputs.pose5_scene(3, noise_px=0.0)
    r = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=z["p0"],
                      p1=truth["p_clean"]).track(start=z["start"])
    fin = r["x"][(r["status"] & 0x7F) == oracle.FINITE]
    xt = truth["x_true"]
    d = np.max(np.abs(fin - xt), axis=1) / np.max(np.abs(xt))
    assert np.min(d) < 1e-8


def test_two_view_start_set():
    """Two-view triangulation (Sec. 4, Eq. constraints, 5 x 5): 8 distinct
    start solutions at p0, each a root; the zero correction is an exact root
    of noise-free consistent data (tested above for the pinned endpoint)."""
    fam = inputs.triangulation_family(2)
    z = np.load(os.path.join(STARTS, "triangulation2.npz"))
    S = z["start"]
    assert S.shape == (8, 5) and distinct(S, 1e-6) == 8
    for x in S:
        assert np.max(np.abs(monodromy.residual(fam.system, x, z["p0"]))) < 1e-10

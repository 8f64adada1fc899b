"""GPU parity of the dense total-degree tracker against the FP64 oracle.

Both sides get the same seeded systems; the GPU runs through the C-ABI.
Bar: status counts per class exactly equal, endpoints matched bijectively
within 1e-8 relative (infinity norm) after the final FP64 refinement.
"""
import numpy as np
import pytest

import oracle
from hcmatch import same_set, match, distinct, rel_dist

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc as mod
    return mod


def _run(hc, n, d, seeds, precision):
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(n, d, seeds)
    gamma = inputs.unit_gamma(seeds[0])
    pr = hc.Problem(base, gamma=gamma, settings=dict(precision=precision))
    b = pr.track(n_instances=len(seeds), coef=coefs).wait()
    return base, coefs, gamma, b


def _oracle(base, coef, gamma, **kw):
    return oracle.OracleProblem(base, gamma=gamma, coef=coef).track(**kw)


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "df"])
@pytest.mark.parametrize("n,d,seeds", [
    (6, 2, list(range(10))),        # the n = 6 quadratic workload, 10 systems
    (1, 2, [3, 4]), (2, 2, [5]), (3, 2, [6, 7]), (5, 2, [8]), (7, 2, [9]),
    (8, 2, [100]), (2, 3, [11]), (3, 3, [12]), (4, 3, [13]), (6, 3, [14]),
])
def test_dense_matches_oracle(hc, n, d, seeds, precision):
    base, coefs, gamma, b = _run(hc, n, d, seeds, precision)
    assert b.result["paths"] == len(seeds) * d ** n
    for s in range(len(seeds)):
        ref = _oracle(base, coefs[s], gamma)
        got = oracle.status_counts(b.status[s])
        want = oracle.status_counts(ref["status"])
        assert got == want, (s, got, want)
        fin_g = (b.status[s] & 0x7F) == oracle.FINITE
        fin_o = (ref["status"] & 0x7F) == oracle.FINITE
        ok, msg = same_set(b.x[s][fin_g], ref["x"][fin_o], TOL)
        assert ok, (s, msg)
        assert np.max(b.be[s][fin_g]) <= 1e-10


@pytest.mark.parametrize("n,d,seed,sample", [(10, 2, 101, 96), (12, 2, 102, 64), (8, 3, 103, 64)])
def test_dense_full_size_sampled(hc, n, d, seed, sample):
    """Full-size systems: every path finite and distinct (Bezout count, a
    property at any size), and sampled oracle paths found among the GPU's."""
    base, coefs, gamma, b = _run(hc, n, d, [seed], 1)
    st = b.status[0]
    assert oracle.status_counts(st)["finite"] == d ** n
    assert distinct(b.x[0], 1e-6) == d ** n
    rng = np.random.default_rng(seed)
    ids = rng.choice(d ** n, size=sample, replace=False)
    ref = _oracle(base, coefs[0], gamma, path_ids=ids)
    assert np.all((ref["status"] & 0x7F) == oracle.FINITE)
    _, dist = match(ref["x"], b.x[0], TOL)
    assert np.max(dist) <= TOL, np.max(dist)


def test_device_pointer_batch_matches_host_batch(hc):
    import torch
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(5, 2, [21, 22, 23])
    gamma = inputs.unit_gamma(21)
    pr = hc.Problem(base, gamma=gamma)
    hb = pr.track(n_instances=3, coef=coefs).wait()
    dev = torch.device("cuda")
    P = pr.paths
    xo = torch.zeros((3, P, 5), dtype=torch.complex128, device=dev)
    so = torch.zeros((3, P), dtype=torch.uint8, device=dev)
    to = torch.zeros((3, P, 3), dtype=torch.int32, device=dev)
    bo = torch.zeros((3, P), dtype=torch.float64, device=dev)
    cf = torch.from_numpy(coefs).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    db = pr.track(n_instances=3, coef=cf, device=True, x_out=xo, status_out=so, steps_out=to,
                  be_out=bo, stream=stream).wait()
    assert np.array_equal(so.cpu().numpy(), hb.status)
    assert np.array_equal(xo.cpu().numpy(), hb.x)
    assert db.result["finite"] == hb.result["finite"] == 3 * 32


def test_summary_counts_match_outputs(hc):
    base, coefs, gamma, b = _run(hc, 4, 2, [31, 32], 1)
    r = b.result
    c = oracle.status_counts(b.status.reshape(-1))
    assert r["finite"] == c["finite"] and r["real"] == c["real"]
    assert r["steps_accepted"] == int(b.steps[..., 0].sum())
    assert r["newton_iters"] == int(b.steps[..., 2].sum())


def test_poll_nonblocking_then_done(hc):
    base, coefs, gamma, _ = _run(hc, 2, 2, [41], 1)
    pr = hc.Problem(base, gamma=gamma)
    bt = pr.track(n_instances=1, coef=coefs)
    code = bt.poll(0)
    assert code in (hc.HC_OK, hc.HC_PENDING)
    assert bt.poll(-1) == hc.HC_OK
    assert bt.result["finite"] == 4


def _golden():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "dense_sweep_oracle.json")
    return json.load(open(path))


@pytest.mark.parametrize("retrack", [2, 0], ids=["retrack_df", "retrack_fp64"])
@pytest.mark.parametrize("ci", range(5), ids=["q8", "q10", "q12", "c6", "c8"])
def test_dense_sweep_matches_oracle_golden(hc, ci, retrack):
    """The benchmarked sweep (16 systems per size class, mixed precision, the
    bench's seeds; the last re-tracking tier in double-float or FP64
    arithmetic) against the oracle's stored outcome on every path
    (tests/golden/dense_sweep_oracle.json):
      - every path the oracle ends at a finite root, the GPU does too;
      - within every system the GPU's finite roots are pairwise distinct
        (so, the oracle's root set being distinct too, the finite sets match);
      - a finite GPU root on a start the oracle fails is a root by the
        oracle's own evaluation (backward error <= 1e-10, cond_1 <= 1e12);
      - sampled starts end within 1e-8 of the oracle's endpoint, tracked live."""
    from paper_2112_03444_gb300 import inputs
    w = inputs.dense_sweep(0)[ci]
    g = _golden()["classes"][ci]
    assert (g["n"], g["d"]) == (w["n"], w["d"])
    pr = hc.Problem(w["base"], gamma=w["gamma"], settings=dict(retrack_precision=retrack))
    b = pr.track(n_instances=len(w["seeds"]), coef=w["coefs"]).wait()
    P = w["d"] ** w["n"]
    for s, gs in enumerate(g["systems"]):
        assert gs["seed"] == w["seeds"][s]
        assert gs["distinct_finite"] == gs["counts"]["finite"]
        fin = (b.status[s] & 0x7F) == hc.PATH_FINITE
        ofin = np.ones(P, bool)
        for p, _ in gs["not_finite"]:
            ofin[p] = False
        assert not np.any(ofin & ~fin), (s, np.nonzero(ofin & ~fin)[0])
        assert distinct(b.x[s][fin]) == int(fin.sum()), s
        extra = np.nonzero(fin & ~ofin)[0]
        if len(extra):
            op = oracle.OracleProblem(w["base"], gamma=w["gamma"], coef=w["coefs"][s])
            for p in extra:
                assert op.backward_error(b.x[s][p]) <= 1e-10, (s, int(p))
                assert op.cond1(b.x[s][p]) <= 1e12, (s, int(p))
    rng = np.random.default_rng(ci)
    ids = rng.choice(P, size=min(24, P), replace=False)
    ref = _oracle(w["base"], w["coefs"][0], w["gamma"], path_ids=ids)
    rf = (ref["status"] & 0x7F) == oracle.FINITE
    assert np.max(rel_dist(b.x[0][ids][rf], ref["x"][rf]), initial=0.0) <= TOL

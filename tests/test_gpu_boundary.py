"""The batch boundary beyond plain tracking: a device step budget reported
by hc_poll as HC_ERR_TIMEOUT, per-instance start subsets, and admission
under a device-memory cap (HC_ERR_BUSY, or waiting with HC_BLOCKING_ADMIT).
All through the C-ABI; every failure is made on the host or through the
inputs, none on the device."""
import os

import numpy as np
import pytest

import oracle
from hcmatch import rel_dist, same_set

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


def test_step_budget_stops_new_paths_and_reports_timeout(hc):
    """64 systems of 256 paths: more paths than the launch has lane groups, so
    with a budget of one step every path not started by the first round of
    fetches stays HC_PATH_NONE, and hc_poll returns HC_ERR_TIMEOUT.  The
    paths that did run are complete and match the oracle."""
    from paper_2112_03444_gb300 import inputs
    seeds = list(range(900, 964))
    base, coefs = inputs.dense_batch(8, 2, seeds)
    g = inputs.unit_gamma(seeds[0])
    pr = hc.Problem(base, gamma=g)
    b = pr.track(n_instances=len(seeds), coef=coefs, step_budget=1)
    assert b.poll(-1) == hc.HC_ERR_TIMEOUT
    r = b.result
    st = b.status
    assert r["untracked"] == int((st == 0).sum()) > 0
    assert r["untracked"] <= 64 * 256 - 1
    started = st != 0
    assert r["steps_total"] >= 1
    # the started paths finished their whole pipeline: compare a few with the oracle
    for s in (0, 63):
        ids = np.nonzero(started[s])[0][:8]
        if len(ids) == 0:
            continue
        ref = oracle.OracleProblem(base, gamma=g, coef=coefs[s]).track(path_ids=ids)
        assert np.array_equal(st[s][ids] & 0x7F, ref["status"] & 0x7F)
        fin = (ref["status"] & 0x7F) == oracle.FINITE
        assert np.max(rel_dist(b.x[s][ids][fin], ref["x"][fin]), initial=0) <= TOL
    # a budget that is never reached changes nothing
    full = pr.track(n_instances=2, coef=coefs[:2]).wait()
    big = pr.track(n_instances=2, coef=coefs[:2], step_budget=10 ** 12)
    assert big.poll(-1) == hc.HC_OK
    assert big.result["untracked"] == 0
    assert np.array_equal(big.status, full.status)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_start_subset_matches_full_batch(hc, precision):
    """Per-instance subsets of the start paths give the full batch's results
    on those paths (bit for bit in FP64, where nothing is re-tracked)."""
    from paper_2112_03444_gb300 import inputs
    seeds = [911, 912, 913]
    base, coefs = inputs.dense_batch(6, 2, seeds)
    g = inputs.unit_gamma(seeds[0])
    pr = hc.Problem(base, gamma=g, settings=dict(precision=precision))
    full = pr.track(n_instances=3, coef=coefs).wait()
    rng = np.random.default_rng(5)
    ids = np.stack([rng.choice(64, size=20, replace=False) for _ in range(3)])
    sub = pr.track(n_instances=3, coef=coefs, path_ids=ids).wait()
    assert sub.status.shape == (3, 20) and sub.x.shape == (3, 20, 6)
    assert sub.result["paths"] == 60
    for k in range(3):
        assert np.array_equal(sub.status[k], full.status[k][ids[k]])
        fin = (sub.status[k] & 0x7F) == hc.PATH_FINITE
        if precision == 0:
            assert np.array_equal(sub.x[k][fin], full.x[k][ids[k]][fin])
        else:
            assert np.max(rel_dist(sub.x[k][fin], full.x[k][ids[k]][fin])) <= TOL


def test_parameter_start_subset_matches_oracle(hc):
    """A subset of the triangulation start set per instance, against the
    oracle tracking the same starts."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1 = np.stack([inputs.triangulation_scene(s)[0] for s in (81, 82)])
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"])
    ids = np.stack([np.arange(0, 294, 7), np.arange(3, 297, 7)])   # 42 starts each
    b = pr.track(n_instances=2, p1=p1, path_ids=ids).wait()
    for k in range(2):
        ref = oracle.OracleProblem(fam.system, kind=oracle.KIND_PARAMETER, p0=z["p0"],
                                   p1=p1[k]).track(start=z["start"][ids[k]])
        assert oracle.status_counts(b.status[k]) == oracle.status_counts(ref["status"])
        fg = (b.status[k] & 0x7F) == hc.PATH_FINITE
        fo = (ref["status"] & 0x7F) == oracle.FINITE
        ok, msg = same_set(b.x[k][fg], ref["x"][fo], TOL)
        assert ok, (k, msg)


def test_subset_rejects_out_of_range_ids(hc):
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(3, 2, [921])
    pr = hc.Problem(base, gamma=inputs.unit_gamma(921))
    with pytest.raises(hc.HCError) as e:
        pr.track(n_instances=1, coef=coefs, path_ids=np.array([[0, 8]]))
    assert e.value.code == hc.HC_ERR_INVALID


def test_memory_cap_refuses_or_waits(hc):
    """Under a cap smaller than any batch, a batch is admitted only when
    nothing else is in flight: a second batch behind a running one gets
    HC_ERR_BUSY, or with HC_BLOCKING_ADMIT waits for it and then runs."""
    import torch
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(6, 2, [931, 932])
    g = inputs.unit_gamma(931)
    pr = hc.Problem(base, gamma=g)
    ref = pr.track(n_instances=2, coef=coefs).wait()
    s = torch.cuda.Stream()
    hc.set_memory_cap(1)
    try:
        with torch.cuda.stream(s):
            torch.cuda._sleep(200_000_000)      # keeps the first batch in flight (~0.1 s)
        first = pr.track(n_instances=2, coef=coefs, stream=s.cuda_stream)
        with pytest.raises(hc.HCError) as e:
            pr.track(n_instances=2, coef=coefs, stream=s.cuda_stream)
        assert e.value.code == hc.HC_ERR_BUSY
        second = pr.track(n_instances=2, coef=coefs, stream=s.cuda_stream, blocking=True)
        assert first.poll(0) == hc.HC_OK          # admission waited for it
        second.wait()
        for b in (first, second):
            assert np.array_equal(b.status, ref.status)
    finally:
        hc.set_memory_cap(0)
    # without a cap nothing is refused
    a = pr.track(n_instances=2, coef=coefs)
    b = pr.track(n_instances=2, coef=coefs)
    a.wait()
    b.wait()

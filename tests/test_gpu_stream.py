"""Continuous admission (hc_stream_*): instances submitted one by one into a
resident tracking launch give, path for path, the results hc_track_batch
gives on the same inputs (statuses and step counts equal, endpoints equal),
with more submissions than slots so that slots are reused while the launch
runs, and with requests arriving while earlier ones are still tracking."""
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STARTS = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc as mod
    return mod


def _same(res, ref_x, ref_st, ref_steps):
    x, st, steps, _ = res
    assert np.array_equal(st, ref_st)
    assert np.array_equal(steps, ref_steps)
    fin = (st & 0x7F) == 1
    assert np.array_equal(x[fin], ref_x[fin])


@pytest.mark.parametrize("n,d,slots", [(6, 2, 4), (4, 3, 2), (8, 2, 3)])
def test_stream_matches_batch_dense(hc, n, d, slots):
    from paper_2112_03444_gb300 import inputs
    seeds = list(range(500 + n, 500 + n + 7))
    base, coefs = inputs.dense_batch(n, d, seeds)
    gamma = inputs.unit_gamma(seeds[0])
    pr = hc.Problem(base, gamma=gamma)
    ref = pr.track(n_instances=len(seeds), coef=coefs).wait()
    s = hc.Stream(pr, slots=slots, idle_us=5000)
    try:
        pending = []
        for i in range(len(seeds)):
            while True:
                try:
                    pending.append((i, s.submit(coef=coefs[i])))
                    break
                except hc.HCError:  # every slot busy: collect the oldest
                    j, tk = pending.pop(0)
                    _same(s.poll(tk), ref.x[j], ref.status[j], ref.steps[j])
        for j, tk in pending:
            _same(s.poll(tk), ref.x[j], ref.status[j], ref.steps[j])
    finally:
        s.close()


def test_stream_matches_batch_triangulation(hc):
    """A parameter family whose paths often take the re-tracking tiers."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1 = np.array([inputs.triangulation_scene(s, views=4)[0] for s in range(40, 46)])
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"])
    ref = pr.track(n_instances=len(p1), p1=p1).wait()
    s = hc.Stream(pr, slots=8, idle_us=5000)
    try:
        tickets = [s.submit(p1=p1[i]) for i in range(len(p1))]
        for i, tk in enumerate(tickets):
            _same(s.poll(tk), ref.x[i], ref.status[i], ref.steps[i])
    finally:
        s.close()


def test_stream_restarts_after_idle_and_times_out_politely(hc):
    """The resident launch leaves after idle_us without work; a later submit
    starts it again.  A zero-timeout poll of a request in flight returns
    None (HC_ERR_TIMEOUT) rather than blocking."""
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(8, 3, [901, 902])
    pr = hc.Problem(base, gamma=inputs.unit_gamma(901))
    ref = pr.track(n_instances=2, coef=coefs).wait()
    s = hc.Stream(pr, slots=2, idle_us=2000)
    try:
        t0 = s.submit(coef=coefs[0])
        assert s.poll(t0, timeout_us=0) is None  # 6561 paths: not done at once
        _same(s.poll(t0), ref.x[0], ref.status[0], ref.steps[0])
        time.sleep(0.05)  # the launch has left (idle)
        t1 = s.submit(coef=coefs[1])
        _same(s.poll(t1), ref.x[1], ref.status[1], ref.steps[1])
        with pytest.raises(hc.HCError):
            s.poll(t1)  # collected already
    finally:
        s.close()


def test_stream_coefficient_family_and_fp64_last_tier(hc):
    """Coefficient interpolation (per-slot staged dc tables) and a stream
    whose last re-tracking tier runs in FP64: still path for path equal to
    the batch on the same settings."""
    from paper_2112_03444_gb300 import inputs
    fam = inputs.p3p_family()
    z = np.load(os.path.join(STARTS, "p3p.npz"))
    rng = np.random.default_rng(3)
    P = len(z["p0"])
    p1 = rng.normal(size=(5, P)) + 1j * rng.normal(size=(5, P))
    for kind, settings in ((hc.HC_COEFFICIENT, None), (hc.HC_PARAMETER, dict(retrack_precision=0))):
        pr = hc.Problem(fam.system, kind=kind, p0=z["p0"], start=z["start"], settings=settings)
        ref = pr.track(n_instances=len(p1), p1=p1).wait()
        s = hc.Stream(pr, slots=2, idle_us=5000)
        try:
            for i in range(len(p1)):
                tk = s.submit(p1=p1[i])
                _same(s.poll(tk), ref.x[i], ref.status[i], ref.steps[i])
        finally:
            s.close()


def test_stream_destroy_with_requests_in_flight(hc):
    """Destroying a stream whose resident launch still has published work
    returns: the stop word ends the launch after the paths in progress."""
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(8, 3, [911, 912, 913])
    pr = hc.Problem(base, gamma=inputs.unit_gamma(911))
    s = hc.Stream(pr, slots=4, idle_us=2000)
    for i in range(3):
        s.submit(coef=coefs[i])
    t0 = time.perf_counter()
    s.close()
    assert time.perf_counter() - t0 < 30.0
    # the problem (and the device) stay usable
    b = pr.track(n_instances=1, coef=coefs[:1]).wait()
    assert (b.status[0] & 0x7F == 1).sum() > 0


def test_stream_rejects_other_precisions(hc):
    from paper_2112_03444_gb300 import inputs
    base, _ = inputs.dense_batch(3, 2, [1])
    pr = hc.Problem(base, settings=dict(precision=hc.HC_PREC_FP64))
    with pytest.raises(hc.HCError):
        hc.Stream(pr, slots=2)

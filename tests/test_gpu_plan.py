"""Plans (hc_plan_create / hc_plan_run): a batch size replayed as a CUDA graph
gives exactly what hc_track_batch gives for the same inputs."""
import os

import numpy as np
import pytest

import oracle
from hcmatch import same_set

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


def _same(a, b):
    assert np.array_equal(a.status, b.status)
    assert np.array_equal(a.steps, b.steps)
    fin = np.isfinite(a.x).all(axis=-1)
    assert np.array_equal(fin, np.isfinite(b.x).all(axis=-1))
    assert np.array_equal(a.x[fin], b.x[fin])
    for k in ("finite", "real", "diverged", "singular", "failed", "escalated",
              "steps_accepted", "steps_rejected", "newton_iters"):
        assert a.result[k] == b.result[k], k


def test_dense_plan_replays_match_track_batch(hc):
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(6, 2, [301, 302, 303, 304, 305, 306])
    g = inputs.unit_gamma(301)
    pr = hc.Problem(base, gamma=g)
    plan = pr.plan(3)
    for sl in (slice(0, 3), slice(3, 6), slice(0, 3)):
        a = plan.run(coef=coefs[sl]).wait()
        b = pr.track(n_instances=3, coef=coefs[sl]).wait()
        _same(a, b)
        # the graph's timing events are recorded on every replay
        assert a.result["device_ms"] > 0 and a.result["track_ms"] > 0
    # coef = NULL: every instance takes the problem's own coefficients
    a = plan.run().wait()
    b = pr.track(n_instances=3).wait()
    _same(a, b)
    ref = oracle.OracleProblem(base, gamma=g).track()
    for i in range(3):
        fin = (a.status[i] & 0x7F) == hc.PATH_FINITE
        rfin = (ref["status"] & 0x7F) == oracle.FINITE
        ok, msg = same_set(a.x[i][fin], ref["x"][rfin], 1e-8)
        assert ok, (i, msg)
    plan.close()


def test_parameter_plan_matches_track_batch(hc):
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"])
    p1 = np.stack([inputs.triangulation_scene(s)[0] for s in (71, 72)])
    plan = pr.plan(2)
    for _ in range(2):
        a = plan.run(p1=p1).wait()
        b = pr.track(n_instances=2, p1=p1).wait()
        _same(a, b)
        assert a.result["finite"] > 400
    plan.close()


def test_runs_on_two_streams_are_ordered(hc):
    """Two runs of one plan enqueued back to back on different streams share
    the plan's buffers; each must still return its own instance's roots."""
    import torch
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(5, 2, [311, 312])
    g = inputs.unit_gamma(311)
    pr = hc.Problem(base, gamma=g)
    plan = pr.plan(1)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    r1 = plan.run(coef=coefs[0:1], stream=s1.cuda_stream)
    r2 = plan.run(coef=coefs[1:2], stream=s2.cuda_stream)
    r2.wait()
    r1.wait()
    for r, sl in ((r1, slice(0, 1)), (r2, slice(1, 2))):
        _same(r, pr.track(n_instances=1, coef=coefs[sl]).wait())
    plan.close()


def test_plan_device_buffers_and_size_check(hc):
    import torch
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(4, 3, [321, 322])
    g = inputs.unit_gamma(321)
    pr = hc.Problem(base, gamma=g)
    plan = pr.plan(2)
    dev = torch.device("cuda:0")
    P, n = pr.paths, pr.n
    c = torch.from_numpy(np.ascontiguousarray(coefs)).to(dev)
    x = torch.zeros((2, P, n), dtype=torch.complex128, device=dev)
    st = torch.zeros((2, P), dtype=torch.uint8, device=dev)
    steps = torch.zeros((2, P, 3), dtype=torch.int32, device=dev)
    be = torch.zeros((2, P), dtype=torch.float64, device=dev)
    a = plan.run(coef=c, x_out=x, status_out=st, steps_out=steps, be_out=be, device=True).wait()
    b = pr.track(n_instances=2, coef=coefs).wait()
    assert np.array_equal(st.cpu().numpy(), b.status)
    fin = (b.status & 0x7F) == hc.PATH_FINITE
    assert np.array_equal(x.cpu().numpy()[fin], b.x[fin])
    assert a.result["finite"] == b.result["finite"]
    with pytest.raises(ValueError):
        plan.run(coef=coefs[:1])
    # the library itself refuses a batch whose size differs from the plan's
    d, _ = pr._desc(1, coefs[:1], None, None, None, None, None, None, False)
    import ctypes
    h = ctypes.c_void_p()
    assert hc._lib.hc_plan_run(plan.h, ctypes.byref(d), ctypes.byref(h)) == hc.HC_ERR_INVALID
    plan.close()

"""Autotuner and the one-path-per-warp kernel variants."""
import os

import numpy as np
import pytest

import oracle
from oracle import KIND_PARAMETER, OracleProblem
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


def test_wide_lane_variants_compute_the_same_paths(hc):
    """One path per warp (lanes = 32) runs each path's arithmetic exactly as
    the default group width does: with re-tracking off (so no path is
    repaired by the FP64 kernel) both give the same statuses and endpoints."""
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(6, 2, [95, 96])
    g = inputs.unit_gamma(95)
    out = []
    for lanes in (0, 32):
        pr = hc.Problem(base, gamma=g, settings=dict(lanes=lanes, escalate=0))
        out.append(pr.track(n_instances=2, coef=coefs).wait())
    assert np.array_equal(out[0].status, out[1].status)
    assert np.max(np.abs(out[0].x - out[1].x)) <= 1e-12 * np.max(np.abs(out[0].x))
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1 = inputs.triangulation_scene(62)[0][None, :]
    out = []
    for lanes in (0, 32):
        pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"],
                        settings=dict(lanes=lanes, escalate=0))
        out.append(pr.track(n_instances=1, p1=p1).wait())
    assert np.array_equal(out[0].status, out[1].status)
    fin = (out[0].status & 0x7F) == hc.PATH_FINITE
    assert fin.sum() > 200
    assert np.max(np.abs(out[0].x[fin] - out[1].x[fin])) <= 1e-12 * np.max(np.abs(out[0].x[fin]))


def test_wide_lane_dense_variant_matches_oracle(hc):
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(6, 2, [91, 92])
    g = inputs.unit_gamma(91)
    pr = hc.Problem(base, gamma=g, settings=dict(lanes=32))
    b = pr.track(n_instances=2, coef=coefs).wait()
    for s in range(2):
        ref = oracle.OracleProblem(base, gamma=g, coef=coefs[s]).track()
        assert oracle.status_counts(b.status[s]) == oracle.status_counts(ref["status"])
        ok, msg = same_set(b.x[s], ref["x"], 1e-8)
        assert ok, msg


def test_wide_lane_parameter_variant_matches_oracle(hc):
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    p1 = inputs.triangulation_scene(61)[0]
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"],
                    settings=dict(lanes=32))
    b = pr.track(n_instances=1, p1=p1[None, :]).wait()
    ref = OracleProblem(fam.system, kind=KIND_PARAMETER, p0=z["p0"], p1=p1).track(start=z["start"])
    assert oracle.status_counts(b.status[0]) == oracle.status_counts(ref["status"])
    fg = (b.status[0] & 0x7F) == oracle.FINITE
    fo = (ref["status"] & 0x7F) == oracle.FINITE
    ok, msg = same_set(b.x[0][fg], ref["x"][fo], 1e-8)
    assert ok, msg


def test_autotune_keeps_fp64_recovery(hc):
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(7, 2, [93, 94])
    pr = hc.Problem(base, gamma=inputs.unit_gamma(93))
    rep = pr.autotune(n_instances=2, coef=coefs)
    assert len(rep["ms"]) >= 3 and all(m > 0 for m in rep["ms"])
    assert rep["tried"][0]["precision"] == hc.HC_PREC_FP64
    assert rep["finite"][rep["best"]] >= rep["finite"][0] == 2 * 128
    b = pr.track(n_instances=2, coef=coefs).wait()
    assert b.result["finite"] == 256


@pytest.mark.parametrize("block", [32, 64])
def test_block_size_does_not_change_the_paths(hc, block):
    """Paths per block (block_threads) only regroups lane groups into blocks:
    with re-tracking off, every path's statuses and endpoints are the same
    bit for bit."""
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(8, 3, [97])
    g = inputs.unit_gamma(97)
    out = []
    for bt in (0, block):
        pr = hc.Problem(base, gamma=g, settings=dict(block_threads=bt, escalate=0))
        out.append(pr.track(n_instances=1, coef=coefs).wait())
    assert np.array_equal(out[0].status, out[1].status)
    assert np.array_equal(out[0].x, out[1].x, equal_nan=True)


def test_autotune_cache_roundtrip(hc, tmp_path):
    """hc_autotune_cached: the first call tunes (block and lane axes included)
    and writes the choice under the problem's shape key; a second problem of
    the same shape takes it from the file without tracking; a malformed file
    is refused."""
    import json
    from paper_2112_03444_gb300 import inputs
    base, coefs = inputs.dense_batch(8, 2, [98, 99])
    cache = tmp_path / "tune.json"
    pr = hc.Problem(base, gamma=inputs.unit_gamma(98))
    rep = pr.autotune(n_instances=2, coef=coefs, cache=cache)
    assert not rep["cached"] and len(rep["ms"]) >= 5
    assert {t["block_threads"] for t in rep["tried"][1:]} >= {64, 128}
    doc = json.loads(cache.read_text())
    (key, entry), = doc.items()
    assert "n=8" in key and "deg=2" in key
    assert entry["block_threads"] == rep["tried"][rep["best"]]["block_threads"]
    pr2 = hc.Problem(base, gamma=inputs.unit_gamma(98))
    rep2 = pr2.autotune(n_instances=2, coef=coefs, cache=cache)
    assert rep2["cached"] and rep2["ms"] == []
    assert pr2.settings.block_threads == entry["block_threads"]
    assert pr2.settings.lanes == entry["lanes"]
    b = pr2.track(n_instances=2, coef=coefs).wait()
    assert b.result["finite"] == 2 * 256
    bad = tmp_path / "bad.json"
    bad.write_text('{"kind=0 n=8 deg=2 terms=360 params=0 sym=1 prec=1": {"lanes": ')
    with pytest.raises(hc.HCError):
        hc.Problem(base, gamma=inputs.unit_gamma(98)).autotune(n_instances=2, coef=coefs,
                                                               cache=bad)

"""The allocation-free tracking entry point against the allocating one.

hc_track_dense_noalloc serves callers that cannot allocate device memory
when they track (an arena that owns the device, a real-time loop that must
not enter the CUDA allocator): its scratch is a fixed device array inside
the library.  Here it is called through the C-ABI twice in a row, on
different shapes so that the second call runs on the first call's leftover
scratch, and each result is compared with hc_track_batch on the same inputs.
"""
import numpy as np
import pytest

from hcmatch import same_set

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc, inputs
    return torch, hc, inputs


def _compare(env, n, d, seeds, settings=None):
    torch, hc, inputs = env
    dev = torch.device("cuda")
    base, coefs = inputs.dense_batch(n, d, seeds)
    gamma = inputs.unit_gamma(seeds[0])
    I = len(seeds)
    P = d ** n
    # allocating entry point
    pr = hc.Problem(base, gamma=gamma, settings=settings)
    ref = pr.track(n_instances=I, coef=coefs).wait()
    # allocation-free entry point, device buffers owned by the caller
    cf = torch.from_numpy(np.ascontiguousarray(coefs)).to(dev)
    xo = torch.zeros((I, P, n), dtype=torch.complex128, device=dev)
    so = torch.zeros((I, P), dtype=torch.uint8, device=dev)
    to = torch.zeros((I, P, 3), dtype=torch.int32, device=dev)
    bo = torch.zeros((I, P), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rc = hc.track_dense_noalloc(n, d, gamma, pr.settings, I, cf, xo, so, to, bo,
                                stream.cuda_stream)
    assert rc == hc.HC_OK, hc._lib.hc_last_error()
    stream.synchronize()
    st = so.cpu().numpy()
    x = xo.cpu().numpy()
    assert np.array_equal(st, ref.status)
    for s in range(I):
        fin = (st[s] & 0x7F) == hc.PATH_FINITE
        ok, msg = same_set(x[s][fin], ref.x[s][fin], TOL)
        assert ok, (n, d, s, msg)


def test_no_alloc_matches_allocating_entry_point_twice(env):
    _compare(env, 6, 2, [201, 202, 203])
    _compare(env, 3, 3, [204, 205])


def test_no_alloc_all_fp64(env):
    # precision FP64: one all-FP64 tracking launch, no escalation lists
    _, hc, _ = env
    _compare(env, 4, 2, [211, 212], dict(precision=hc.HC_PREC_FP64))


def test_no_alloc_mixed_without_escalation(env):
    # mixed without re-tracking: the escalation, duplicate and restart
    # buffers are absent and failed FP32 paths stay failed
    _, hc, _ = env
    _compare(env, 4, 2, [213, 214], dict(escalate=0))
    _compare(env, 3, 3, [215, 216], dict(escalate=0))


def test_no_alloc_double_float(env):
    # precision DF: the double-float kernel (one path per warp) and its table
    _, hc, _ = env
    _compare(env, 4, 2, [217, 218], dict(precision=hc.HC_PREC_DF))
    _compare(env, 3, 3, [219], dict(precision=hc.HC_PREC_DF))


def test_no_alloc_fp64_last_tier(env):
    # mixed with the last re-tracking tier in FP64 rather than double-floats
    _, hc, _ = env
    _compare(env, 6, 2, [220, 221], dict(retrack_precision=hc.HC_PREC_FP64))


def test_no_alloc_rejects_batches_beyond_its_scratch(env):
    torch, hc, inputs = env
    dev = torch.device("cuda")
    n, d, I = 8, 3, 400      # 400 * 6561 paths: far beyond the fixed array
    cf = torch.zeros(1, dtype=torch.complex128, device=dev)
    rc = hc.track_dense_noalloc(n, d, 1.0, None, I, cf, cf, cf, cf)
    assert rc == hc.HC_ERR_INVALID
    assert b"scratch" in hc._lib.hc_last_error()

"""The standalone batched solver (hc_batched_solve, paper Sec. 6 / Fig. 3)
against the oracle's augmented-matrix LU solve and numpy, on seeded random
complex systems of every size 1..32, with batches that leave ragged blocks."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc
    return torch, hc


def _systems(n, batch, seed):
    rng = np.random.default_rng([seed, n, batch])
    A = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    b = rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))
    return A, b


def _solve(env, A, b, fp32):
    torch, hc = env
    dt = torch.complex64 if fp32 else torch.complex128
    Ad = torch.from_numpy(A).to("cuda", dt)
    bd = torch.from_numpy(b).to("cuda", dt)
    x = torch.zeros_like(bd)
    info = torch.full((A.shape[0],), -7, dtype=torch.int32, device="cuda")
    assert hc.batched_solve(Ad, bd, x, info) == hc.HC_OK
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), info.cpu().numpy()


@pytest.mark.parametrize("fp32", [0, 1], ids=["z", "c"])
@pytest.mark.parametrize("n", list(range(1, 33)))
def test_batched_solve_matches_oracle_and_numpy(env, n, fp32):
    batch = 37 + 3 * n                      # not a multiple of any block's system count
    A, b = _systems(n, batch, 1)
    x, info = _solve(env, A, b, fp32)
    assert np.all(info == 0)
    want = np.linalg.solve(A, b[..., None])[..., 0]
    cond = np.linalg.cond(A)
    err = np.max(np.abs(x - want), axis=1) / np.max(np.abs(want), axis=1)
    # backward-stable elimination: error <= c * n * cond * unit roundoff
    u = 2.0 ** -24 if fp32 else 2.0 ** -53
    assert np.all(err <= 64 * n * cond * u), float(np.max(err / (n * cond * u)))
    for k in (0, batch - 1):                 # the oracle's own solve, first and last system
        xo, ok = oracle.solve(A[k], b[k])
        assert ok
        assert np.max(np.abs(x[k] - xo)) / np.max(np.abs(xo)) <= 64 * n * cond[k] * u


def test_batched_solve_flags_singular_systems(env):
    A, b = _systems(6, 64, 3)
    A[5] = 0.0                                # zero matrix
    A[9][:, 2] = 0.0                          # a zero column
    x, info = _solve(env, A, b, 0)
    assert info[5] == 1 and info[9] == 1
    good = np.setdiff1d(np.arange(64), [5, 9])
    assert np.all(info[good] == 0)
    want = np.linalg.solve(A[good], b[good][..., None])[..., 0]
    assert np.max(np.abs(x[good] - want) / np.max(np.abs(want), axis=1, keepdims=True)) < 1e-10


def test_batched_solve_needs_pivoting(env):
    """Leading zeros on the diagonal: no solution without row interchanges."""
    A, b = _systems(5, 40, 4)
    A[:, 0, 0] = 0.0
    A[:, 1, 1] = 0.0
    x, info = _solve(env, A, b, 0)
    assert np.all(info == 0)
    want = np.linalg.solve(A, b[..., None])[..., 0]
    assert np.max(np.abs(x - want) / np.max(np.abs(want), axis=1, keepdims=True)) < 1e-10


def test_batched_solve_argument_checks(env):
    torch, hc = env
    lib = hc._lib
    assert lib.hc_batched_solve(0, 1, 0, None, None, None, None, None) == hc.HC_ERR_INVALID
    assert lib.hc_batched_solve(33, 1, 0, None, None, None, None, None) == hc.HC_ERR_INVALID
    assert lib.hc_batched_solve(4, 0, 0, None, None, None, None, None) == hc.HC_OK


def test_batched_solve_large_batch(env):
    """A batch far larger than one wave of blocks (the grid strides)."""
    A, b = _systems(8, 200_003, 5)
    x, info = _solve(env, A, b, 1)
    assert np.all(info == 0)
    idx = np.random.default_rng(0).choice(len(A), 500, replace=False)
    want = np.linalg.solve(A[idx], b[idx][..., None])[..., 0]
    cond = np.linalg.cond(A[idx])
    err = np.max(np.abs(x[idx] - want), axis=1) / np.max(np.abs(want), axis=1)
    assert np.all(err <= 64 * 8 * cond * 2.0 ** -24)

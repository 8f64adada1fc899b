"""Continuous-batching server: each request's result is the same alone and
in a mix of concurrently running requests of different problems, and the mix
is really batched and overlapped on the device."""
import os
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STARTS = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_03444_gb300 import hc, inputs
    return hc, inputs


def _problems(hc, inputs):
    probs = {}
    for n in (4, 6, 8):
        base = inputs.dense_system(n, 2, 500 + n)
        probs[f"q{n}"] = (hc.Problem(base, gamma=inputs.unit_gamma(500 + n)),
                          lambda s, n=n: inputs.dense_coefficients(n, 2, s).reshape(-1))
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    probs["tri"] = (hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"]),
                    lambda s: inputs.triangulation_scene(s)[0])
    return probs


def test_results_alone_equal_results_in_the_mix(env):
    hc, inputs = env
    probs = _problems(hc, inputs)
    rng = np.random.default_rng(0)
    reqs = [(k, 900 + i) for i, k in enumerate(rng.choice(sorted(probs), size=40))]
    # mix: submitted from a separate thread at short random intervals while
    # earlier requests run
    srv = hc.Server(n_streams=4, max_batch_instances=16)
    ids = [None] * len(reqs)

    def producer():
        for j, (k, seed) in enumerate(reqs):
            ids[j] = srv.submit(probs[k][0], probs[k][1](seed))
            time.sleep(float(rng.exponential(0.0005)))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    mixed = [srv.wait(ids[j], probs[k][0]) for j, (k, _) in enumerate(reqs)]
    stats = srv.stats()
    srv.close()
    assert stats["done"] == len(reqs)
    assert stats["max_batch_instances"] > 1, stats     # requests were batched
    assert stats["max_inflight_batches"] > 1, stats    # batches overlapped
    # alone: one request per batch, one at a time
    alone_srv = hc.Server(n_streams=1, max_batch_instances=1)
    for j, (k, seed) in enumerate(reqs):
        rid = alone_srv.submit(probs[k][0], probs[k][1](seed))
        x, st, info = alone_srv.wait(rid, probs[k][0])
        xm, stm, infom = mixed[j]
        assert info["batch_instances"] == 1
        assert np.array_equal(st, stm), (k, seed)
        fin = (st & 0x7F) == hc.PATH_FINITE
        assert np.max(np.abs(x[fin] - xm[fin]) / np.maximum(1, np.abs(x[fin]))) <= 1e-8
    alone_srv.close()


def test_server_admission_respects_the_memory_cap(env):
    hc, inputs = env
    base = inputs.dense_system(6, 2, 77)
    pr = hc.Problem(base, gamma=inputs.unit_gamma(77))
    per = hc.problem_query(pr.h)["device_bytes_per_instance"]
    srv = hc.Server(n_streams=4, max_batch_instances=64, max_device_bytes=3 * per)
    ids = [srv.submit(pr, inputs.dense_coefficients(6, 2, s).reshape(-1)) for s in range(24)]
    out = [srv.wait(i, pr) for i in ids]
    stats = srv.stats()
    srv.close()
    assert stats["max_inflight_bytes"] <= 3 * per
    assert stats["max_batch_instances"] <= 3
    assert all(info["finite"] == 64 for _, _, info in out)

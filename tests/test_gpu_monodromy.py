"""Monodromy on the GPU (hc_monodromy_solve, paper Sec. 7): from one seed
solution at the committed generic parameter point p0, the triangle loops
tracked by the GPU must find exactly the committed start set -- the one the
FP64 oracle's monodromy produced (296 solutions for 4-view triangulation)."""
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


def test_gpu_monodromy_reproduces_triangulation_start_set(hc):
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    sols, info = hc.monodromy_solve(fam.system, z["start"][17], z["p0"], seed=3,
                                    stall_loops=10, loops_per_round=4)
    assert len(sols) == len(z["start"]) == 296, (len(sols), info)
    ok, msg = same_set(sols, z["start"], 1e-8)
    assert ok, msg
    # every solution satisfies F(x; p0) = 0 by the oracle's own evaluation
    op = oracle.OracleProblem(fam.system, kind=oracle.KIND_PARAMETER, p0=z["p0"], p1=z["p0"])
    for x in sols[::37]:
        H, _, _ = op.eval(x, 1.0)
        assert np.max(np.abs(H)) < 1e-10
    assert info["loops"] >= 10 and info["paths_tracked"] > 0


def test_gpu_monodromy_rejects_bad_descriptors(hc):
    from paper_2112_03444_gb300 import inputs
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(STARTS, "triangulation4.npz"))
    with pytest.raises(hc.HCError) as e:
        hc.monodromy_solve(fam.system, z["start"][0], z["p0"], stall_loops=0)
    assert e.value.code == hc.HC_ERR_INVALID
    with pytest.raises(hc.HCError) as e:                       # capacity below the count
        hc.monodromy_solve(fam.system, z["start"][0], z["p0"], max_solutions=10,
                           stall_loops=3)
    assert e.value.code == hc.HC_ERR_INVALID


@pytest.mark.parametrize("name,count", [("p3p", 8), ("pose5_depth", 40)])
def test_gpu_monodromy_with_sign_symmetries(hc, name, count):
    """P3P (rho -> -rho) and relative pose with depth (q -> -q): the GPU
    monodromy, adding sign images of every new solution and tracking one
    start per orbit, reproduces the oracle's committed start set."""
    from paper_2112_03444_gb300 import inputs
    fam = {"p3p": inputs.p3p_family, "pose5_depth": inputs.pose5_depth_family}[name]()
    z = np.load(os.path.join(STARTS, f"{name}.npz"))
    sols, info = hc.monodromy_solve(fam.system, z["start"][1], z["p0"], seed=5,
                                    stall_loops=8, loops_per_round=4,
                                    symmetries=fam.sign_masks)
    assert len(sols) == count, (len(sols), info)
    ok, msg = same_set(sols, z["start"], 1e-8)
    assert ok, msg

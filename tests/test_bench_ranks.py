"""Host logic of the N > 1 bench path, on CPU: replicas get disjoint seeded
workloads, rank 0 reports the slowest replica (max over ranks through a
world-size-2 gloo group), and the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(values[rank], world)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(got))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2(tmp_path):
    import torch.multiprocessing as mp
    values = [12.5, 17.25]
    mp.spawn(_rank_main, args=(2, _free_port(), values, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert float(open(tmp_path / f"rank{r}.txt").read()) == max(values)


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_replica_workloads_are_disjoint_and_seeded():
    import bench
    import numpy as np
    w0, w0b, w1 = bench.workload(0), bench.workload(0), bench.workload(1)
    s0 = {s for w in w0 for s in w["seeds"]}
    s1 = {s for w in w1 for s in w["seeds"]}
    assert not (s0 & s1)
    for a, b in zip(w0, w0b):
        assert np.array_equal(a["coefs"], b["coefs"])
    assert [(w["n"], w["d"]) for w in w0] == [(w["n"], w["d"]) for w in w1]


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""

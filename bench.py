"""Benchmark: batched homotopy-continuation path tracking on one GB300.

Workload (the dense total-degree sweep): dense random quadratic systems with
n = 8, 10, 12 unknowns (256 / 1024 / 4096 paths each) and dense random cubic
systems with n = 6, 8 (729 / 6561 paths), complex Gaussian coefficients,
16 systems per size; every path of every system of a size runs in one
persistent mixed-precision launch (FP32 tracking, double-float endgame
residuals and refinement, FP64 re-tracking tiers).  One step = all five size
classes, 202,656 paths.

Prints one JSON line.  value = oracle-matched paths/s: a path counts when the
GPU ends it at a finite root and the FP64 oracle, run once on every path of
the same seeded systems (tests/golden/dense_sweep_oracle.json), ends the same
start at a finite root too, provided the GPU's finite roots of every system
are pairwise distinct (a finite root set of distinct refined roots of a
system whose oracle root set is complete is that root set).  Beside it:
recovery against the oracle's recovery, a sampled endpoint comparison with
the oracle run live, the same sweep as one plain-FP64 launch per system, the
dominant kernel's roofline (FP32 and FP64), per-request latency of a short
serving run, and the oracle's own throughput on the host (all cores and one).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2112_03444_gb300 import inputs  # noqa: E402  (problem data only)

SIZES = list(inputs.DENSE_SWEEP_SIZES)   # (n, degree)
SYSTEMS_PER_SIZE = inputs.DENSE_SWEEP_SYSTEMS
WORKLOAD = "dense total-degree sweep: quadratics n=8,10,12; cubics n=6,8; 16 systems per size"
METRIC = "paths/s and systems/s at oracle-matched roots (1e-8); p50/p99 latency per system"
GOLDEN = os.path.join(ROOT, "tests", "golden", "dense_sweep_oracle.json")
START_DIR = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")


def source_sha() -> str:
    """sha256 (16 hex) of the sources that compile into the dominant tracking
    kernel: its translation unit and the device headers."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2112_03444_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cuh")) + [os.path.join(csrc, "dense_c32.cu")])
    h = hashlib.sha256()
    for f in sorted(files, key=lambda f: os.path.relpath(f, ROOT)):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu capture, or None once the
    kernel sources have changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        kv = dict(l.split(None, 1) for l in open(path).read().splitlines()
                  if l and not l.startswith("#"))
    except (OSError, ValueError):
        return None
    if kv.get("source_sha", "").strip() != source_sha():
        return None
    return int(kv["dram_bytes_per_launch"])


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def max_over_ranks(value, world, device=None):
    """The largest value over the ranks (the slowest replica's step time):
    rank 0 reports whole-job throughput from it.  world <= 1: value."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world, device=None):
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload(rank=0):
    """Per size: dict(n, d, base TermSystem, coefs [16, T], seeds, gamma);
    each replica rank its own seeds."""
    return inputs.dense_sweep(rank)


# ---------------------------------------------------------------- flop model
def dense_flops_per_unit(n, d):
    """Algorithmic complex-FMA counts of one evaluation / solve (dense system).

    E_H = n*M (one cFMA per monomial per equation), E_Ht = E_H (linear
    homotopy in the coefficients), E_Hx = n * sum_m (#distinct variables of m),
    S = sum_{j<n} j(j+1) + n(n+1)/2 (augmented LU + back substitution).
    """
    import itertools
    from math import comb
    M = comb(n + d, d)
    dv = 0
    for deg in range(d + 1):
        for c in itertools.combinations_with_replacement(range(n), deg):
            dv += len(set(c))
    E_H = n * M
    E_Hx = n * dv
    S = sum(j * (j + 1) for j in range(n)) + n * (n + 1) // 2
    return dict(E_H=E_H, E_Ht=E_H, E_Hx=E_Hx, S=S)


def flops(n, d, steps, newton):
    """Flops of `steps` predictor steps (4 RK stages: E_Hx + E_Ht + S each)
    and `newton` corrector iterations (E_H + E_Hx + S each), cFMA = 8 flops."""
    f = dense_flops_per_unit(n, d)
    rk = 4 * (f["E_Hx"] + f["E_Ht"] + f["S"])
    nw = f["E_H"] + f["E_Hx"] + f["S"]
    return 8.0 * (steps * rk + newton * nw)


# ---------------------------------------------------------------- oracle goldens
def load_golden():
    """The oracle's stored outcome on every path of the rank-0 sweep, or None."""
    try:
        return json.load(open(GOLDEN))
    except OSError:
        return None


def nearest_other(x):
    """Relative infinity distance of every row of x to its nearest other row."""
    from scipy.spatial import cKDTree
    if len(x) < 2:
        return np.full(len(x), np.inf)
    emb = np.concatenate([x.real, x.imag], axis=1)
    d, idx = cKDTree(emb).query(emb, k=2, p=np.inf)
    scale = np.maximum(1.0, np.max(np.abs(x), axis=1))
    return d[:, 1] / scale


def match_sweep(wl, statuses, xs, golden, dup_tol=1e-6):
    """Oracle-matched paths of one sweep step (see the module docstring).

    statuses[c] [systems, paths] u8, xs[c] [systems, paths, n] complex.
    matched: paths finite on both sides; oracle_only: paths the oracle ends
    finite and the GPU does not (recovery equals the oracle's iff none);
    gpu_only: finite GPU roots on starts the oracle fails (not counted)."""
    matched = total = oracle_finite = gpu_finite = dup_systems = 0
    oracle_only, gpu_only = [], []
    for ci, w in enumerate(wl):
        gcls = golden["classes"][ci] if golden else None
        for s in range(len(w["seeds"])):
            st = statuses[ci][s] & 0x7F
            fin = st == 1
            total += len(st)
            gpu_finite += int(fin.sum())
            dup = nearest_other(xs[ci][s][fin]).min(initial=np.inf) <= dup_tol
            dup_systems += int(dup)
            if gcls is None:
                matched += 0 if dup else int(fin.sum())
                continue
            g = gcls["systems"][s]
            assert g["seed"] == w["seeds"][s], "golden written for another workload"
            ofin = np.ones(len(st), bool)
            for p, code in g["not_finite"]:
                ofin[p] = False
            oracle_finite += int(ofin.sum())
            if dup:                               # a root reported twice: nothing matches
                fin = np.zeros_like(fin)
            matched += int((fin & ofin).sum())
            oracle_only += [[w["n"], w["d"], s, int(p), int(statuses[ci][s][p])]
                            for p in np.nonzero(ofin & ~fin)[0]]
            gpu_only += [[w["n"], w["d"], s, int(p)] for p in np.nonzero(fin & ~ofin)[0]]
    return dict(matched=matched, total=total, gpu_finite=gpu_finite,
                oracle_finite=oracle_finite if golden else None,
                systems_with_duplicate_roots=dup_systems, oracle_only=oracle_only,
                gpu_only=len(gpu_only))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (a temporary file)."""

    def __init__(self):
        import tempfile
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hc_bench_clocks_{os.getpid()}.csv")

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        dev = os.environ.get("LOCAL_RANK", "0")
        for line in open(self.path).read().splitlines()[1:]:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != dev:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                    samples=len(sm))


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2112_03444_gb300 import hc

    rank, world = env_rank()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    # one stream per size class: the five persistent launches (and their
    # re-tracking launches) overlap on the device
    class_streams = [torch.cuda.Stream(device=dev) for _ in SIZES]
    wl = workload(rank)
    golden = load_golden() if rank == 0 else None
    problems, bufs = [], []
    for w in wl:
        pr = hc.Problem(w["base"], gamma=w["gamma"], settings=dict(precision=hc.HC_PREC_MIXED))
        I, P, n = SYSTEMS_PER_SIZE, pr.paths, w["n"]
        bufs.append(dict(
            coef=torch.from_numpy(w["coefs"]).to(dev),
            x=torch.zeros((I, P, n), dtype=torch.complex128, device=dev),
            st=torch.zeros((I, P), dtype=torch.uint8, device=dev),
            steps=torch.zeros((I, P, 3), dtype=torch.int32, device=dev),
            be=torch.zeros((I, P), dtype=torch.float64, device=dev)))
        problems.append(pr)
    # one captured CUDA graph per size class (staging, tracking launch,
    # re-tracking branch, summary), replayed every step
    plans = [pr.plan(SYSTEMS_PER_SIZE) for pr in problems]
    total_paths = sum(p.paths * SYSTEMS_PER_SIZE for p in problems)
    order = sorted(range(len(wl)), key=lambda i: -problems[i].paths * wl[i]["n"] ** 2)
    total_systems = SYSTEMS_PER_SIZE * len(problems)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        batches = [None] * len(problems)
        ev = torch.cuda.Event()
        ev.record(stream)
        # largest class first: later classes' launches fill the SMs while the
        # earlier ones finish their re-tracking tails
        for i in order:
            b, cs = bufs[i], class_streams[i]
            cs.wait_event(ev)
            batches[i] = plans[i].run(coef=b["coef"], device=True, x_out=b["x"],
                                      status_out=b["st"], steps_out=b["steps"], be_out=b["be"],
                                      stream=cs.cuda_stream)
        for cs in class_streams:
            done = torch.cuda.Event()
            done.record(cs)
            stream.wait_event(done)
        return batches

    for _ in range(args.warmup):
        for bt in step():
            bt.wait()
            bt.close()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler()
    sampler.start()
    step_ms, results = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))           # L2 flush between timed steps (not timed)
            e0.record(stream)
        bts = step()
        with torch.cuda.stream(stream):
            e1.record(stream)
        for bt in bts:
            bt.wait()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        results.append([bt.result for bt in bts])
        # per graph replay: staging, tracking, duplicate check, FP64-residual
        # re-tracking, second duplicate check, all-FP64 re-tracking, summary
        launches += 7 * len(bts)
        for bt in bts:
            bt.close()
    clocks = sampler.stop()
    torch.cuda.synchronize()
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, world, dev)

    # ---- oracle matching of the last timed step
    m = match_sweep(wl, [b["st"].cpu().numpy() for b in bufs],
                    [b["x"].cpu().numpy() for b in bufs], golden)
    matched_all = sum_over_ranks(m["matched"], world, dev)
    recovery = m["matched"] / m["total"]
    oracle_recovery = m["oracle_finite"] / m["total"] if golden else None

    # ---- dominant kernel roofline: the tracking launch of the class with the
    # most algorithmic work in the timed step (from its device step
    # counters), timed alone (inside the step the five classes overlap, so a
    # launch's wall time there includes waiting for SM slots)
    last = results[-1]

    def class_flops(i):
        r = last[i]
        return flops(wl[i]["n"], wl[i]["d"],
                     r["steps_accepted"] + r["steps_rejected"] - r["esc_accepted"] - r["esc_rejected"],
                     r["newton_iters"] - r["esc_newton"])
    dom = max(range(len(wl)), key=class_flops)
    dw, dpr, db = wl[dom], problems[dom], bufs[dom]
    dk_ms, dflop = [], []
    for _ in range(3):
        bt = dpr.track(n_instances=SYSTEMS_PER_SIZE, coef=db["coef"], device=True, x_out=db["x"],
                       status_out=db["st"], steps_out=db["steps"], be_out=db["be"], stream=sp)
        bt.wait()
        r = bt.result
        dk_ms.append(r["track_ms"])
        # flops of the tracking launch only: all steps minus the re-tracking tiers'
        dflop.append(flops(dw["n"], dw["d"],
                           r["steps_accepted"] + r["steps_rejected"] - r["esc_accepted"] - r["esc_rejected"],
                           r["newton_iters"] - r["esc_newton"]))
        bt.close()
    achieved = statistics.mean(f / (m_ * 1e-3) for f, m_ in zip(dflop, dk_ms)) / 1e12
    peak_fp32, _ = hc.measure_fma_peak(False)
    peak_fp64, _ = hc.measure_fma_peak(True)

    # ---- end-to-end through the public API with host buffers: every step
    # copies the coefficients from pinned host memory and reads the endpoints,
    # statuses, step counts and backward errors back into pinned host memory
    # (buffers allocated once, as a serving loop would keep them)
    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()
    hbufs = []
    for w, pr in zip(wl, problems):
        I, P, n = SYSTEMS_PER_SIZE, pr.paths, w["n"]
        c = pinned(w["coefs"].shape, torch.complex128)
        c[...] = w["coefs"]
        hbufs.append(dict(coef=c, x=pinned((I, P, n), torch.complex128),
                          st=pinned((I, P), torch.uint8), steps=pinned((I, P, 3), torch.int32),
                          be=pinned((I, P), torch.float64)))
    e2e_ms = []
    h2d = sum(h["coef"].nbytes for h in hbufs)
    d2h = sum(h["x"].nbytes + h["st"].nbytes + h["steps"].nbytes + h["be"].nbytes for h in hbufs)
    for k in range(max(3, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bts = [plans[i].run(coef=hbufs[i]["coef"], x_out=hbufs[i]["x"], status_out=hbufs[i]["st"],
                            steps_out=hbufs[i]["steps"], be_out=hbufs[i]["be"],
                            stream=class_streams[i].cuda_stream) for i in order]
        for bt in bts:
            bt.wait()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        for bt in bts:
            bt.close()
    e2e_ok = all(np.array_equal(h["st"], b["st"].cpu().numpy()) for h, b in zip(hbufs, bufs))
    e2e = statistics.median(e2e_ms)
    me = match_sweep(wl, [h["st"] for h in hbufs], [h["x"] for h in hbufs], golden)

    # ---- the same sweep as one plain-FP64 launch per system (80 launches on
    # one stream, device buffers): the form the batched mixed-precision
    # launches replace, with its own oracle matching and FP64 roofline
    fp64 = None
    if not args.no_fp64_leg:
        fprobs = [hc.Problem(w["base"], gamma=w["gamma"], settings=dict(precision=hc.HC_PREC_FP64))
                  for w in wl]
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        fbts = []
        for i in order:
            pr, b = fprobs[i], bufs[i]
            for k in range(SYSTEMS_PER_SIZE):
                fbts.append((i, pr.track(n_instances=1, coef=b["coef"][k:k + 1], device=True,
                                         x_out=b["x"][k:k + 1], status_out=b["st"][k:k + 1],
                                         steps_out=b["steps"][k:k + 1], be_out=b["be"][k:k + 1],
                                         stream=sp)))
        s1.record(stream)
        fl64, tr64 = 0.0, 0.0
        for i, bt in fbts:
            bt.wait()
            r = bt.result
            fl64 += flops(wl[i]["n"], wl[i]["d"], r["steps_accepted"] + r["steps_rejected"],
                          r["newton_iters"])
            tr64 += r["track_ms"]
            bt.close()
        torch.cuda.synchronize()
        f_ms = s0.elapsed_time(s1)
        mf = match_sweep(wl, [b["st"].cpu().numpy() for b in bufs],
                         [b["x"].cpu().numpy() for b in bufs], golden)
        ach64 = fl64 / (tr64 * 1e-3) / 1e12
        fp64 = dict(value=mf["matched"] * world / (f_ms * 1e-3), unit="paths/s", ms_per_step=f_ms,
                    recovery=mf["matched"] / mf["total"],
                    recovery_equals_oracle=(mf["matched"] == mf["oracle_finite"]) if golden else None,
                    oracle_only=len(mf["oracle_only"]), gpu_only=mf["gpu_only"],
                    form="one hc_track_batch per system, precision FP64 (all-FP64 kernel), one "
                         "stream, device buffers",
                    roofline=dict(bound="alu", achieved=ach64, peak=peak_fp64 / 1e12,
                                  unit="TFLOP/s", frac=ach64 * 1e12 / peak_fp64,
                                  note="of measured: algorithmic flops of all 80 FP64 tracking "
                                       "launches / their summed launch time, against the FP64 "
                                       "FMA throughput from hc_measure_fma_peak(fp64=1)"))

    # ---- configs 3 and 4 at their scale (extra keys; the headline stays the sweep)
    params = None if args.no_param_legs else param_legs(hc, args)

    # ---- the standalone fused batched solver against cuBLAS (paper Fig. 3)
    solve = None if args.no_solve_leg else solve_leg(hc, torch, stream)

    # ---- a short serving run: per-request latency (Poisson arrivals)
    # The mix without trifocal gives the per-request latency of the line; with
    # trifocal, its batches' all-FP64 re-tracking tails (persistent launches
    # at full occupancy for seconds) hold every SM and the other requests
    # queue behind them (reported beside, at a lower rate).
    serving = serving_tf = None
    if not args.no_serving_leg:
        serving = serve_rows(hc, [args.serve_rate], args.serve_duration, trifocal=False,
                             fp64_requests=0)[0]
        serving_tf = serve_rows(hc, [args.serve_rate / 4], args.serve_duration, trifocal=True,
                                fp64_requests=0)[0]
    # continuous admission into a resident launch against the batch server,
    # single-kind Poisson streams at rising rates (the saturation knee)
    admission = None
    if not args.no_serving_leg and not args.no_admission_leg:
        admission = stream_rows(hc, [float(r) for r in args.admission_rates.split(",")],
                                args.admission_duration)

    line = dict(
        metric=METRIC, value=matched_all / (ms * 1e-3), unit="paths/s",
        systems_per_s=total_systems * world / (ms * 1e-3),
        latency_ms=dict(p50=serving["p50_ms"], p99=serving["p99_ms"],
                        note="per request of the serving leg: Poisson arrivals of dense "
                             "quadratics n = 4..12 and 4-view triangulation, continuous "
                             "batching; with trifocal in the mix see serving_with_trifocal")
        if serving else None,
        n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="c64+c128 (mixed)",
        data="synthetic",
        config=dict(workload=WORKLOAD, paths_per_step=total_paths, systems_per_step=total_systems,
                    precision="mixed: FP32 tracking, double-float endgame residuals and "
                              "refinement, FP64 re-tracking tiers",
                    l2="flushed between timed steps (256 MB write)", parallelism=f"replicas{world}",
                    launch="one captured CUDA graph per size class (hc_plan_run), five streams",
                    matching="rank 0 against the stored FP64 oracle outcome of every path "
                             "(tests/golden/dense_sweep_oracle.json); other replicas: distinct "
                             "finite roots"),
        batch_step_ms=dict(p50=statistics.median(step_ms), p99=float(np.percentile(step_ms, 99))),
        recovery=recovery, oracle_recovery=oracle_recovery,
        recovery_equals_oracle=(m["matched"] == m["oracle_finite"]) if golden else None,
        matched=m, escalated=sum(r["escalated"] for r in last),
        e2e=dict(value=me["matched"] * world / (e2e * 1e-3), unit="paths/s",
                 h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, ms_per_step=e2e,
                 path="hc_plan_run per size class on its own stream, pinned host buffers",
                 same_statuses_as_device_run=e2e_ok),
        gpu_launches=launches,
        one_system_per_launch_fp64=fp64,
        roofline=dict(bound="alu", achieved=achieved, peak=peak_fp32 / 1e12, unit="TFLOP/s",
                      frac=achieved * 1e12 / peak_fp32, traffic=recorded_traffic(),
                      kernel=f"dense_td_kernel<n={dw['n']}, d={dw['d']}, mixed>",
                      kernel_ms=statistics.mean(dk_ms),
                      fp64_peak=peak_fp64 / 1e12,
                      peak_note="of measured: FP32 FMA throughput from hc_measure_fma_peak on "
                                "this GPU in this run; algorithmic flops from the device step "
                                "counters"),
        serving=serving,
        serving_with_trifocal=serving_tf,
        admission=admission,
        batched_solve=solve,
        parameter_workloads=params,
        clocks=clocks,
    )
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"], line["oracle_match"] = cpu_baseline(wl, bufs_host(bufs), args)
        line["cpu_baseline_1thread"], _ = cpu_baseline(wl, None, args, sample=args.cpu_sample_1t,
                                                       threads=1)
    if golden is not None and not line["recovery_equals_oracle"]:
        line["recovery_note"] = ("the GPU does not end every path the oracle solves: see "
                                 "matched.oracle_only")
    if world > 1:
        dist.destroy_process_group()
    return line


def bufs_host(bufs):
    return [dict(x=b["x"].cpu().numpy()) for b in bufs]


# ---------------------------------------------------------------- configs 3 and 4 at scale
def _status_diff(got, want):
    return int(np.sum((np.asarray(got) & 0x7F) != (np.asarray(want) & 0x7F)))


def param_legs(hc, args):
    """4-view triangulation with tri_instances scenes in one batch, and the
    trifocal pose with trifocal_instances scenes in one batch (orbit
    representatives of the quaternion signs), both mixed precision.  Parity:
    two triangulation instances against the FP64 oracle run live on all 296
    starts; the first two trifocal instances are the scenes of the stored
    oracle golden (tests/golden/trifocal_oracle.npz), compared on all 5344
    starts through its endpoint projections."""
    import oracle
    from scipy.spatial import cKDTree
    out = {}
    # ---- 4-view triangulation
    fam = inputs.triangulation_family(4)
    z = np.load(os.path.join(START_DIR, "triangulation4.npz"))
    I = args.tri_instances
    p1 = np.stack([inputs.triangulation_scene(20_000 + k)[0] for k in range(I)])
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"])
    pr.track(n_instances=min(I, 64), p1=p1[:64]).wait()                  # warm-up
    t0 = time.perf_counter()
    b = pr.track(n_instances=I, p1=p1).wait()
    wall = time.perf_counter() - t0
    r = b.result
    checks = []
    for k in (0, I - 1):
        ref = oracle.OracleProblem(fam.system, kind=oracle.KIND_PARAMETER, p0=z["p0"],
                                   p1=p1[k]).track(start=z["start"])
        checks.append(dict(instance=k, status_diffs=_status_diff(b.status[k], ref["status"]),
                           gpu=oracle.status_counts(b.status[k]),
                           oracle=oracle.status_counts(ref["status"])))
    out["triangulation4"] = dict(
        instances=I, paths=r["paths"], device_ms=r["device_ms"], wall_ms=wall * 1e3,
        systems_per_s=I / (r["device_ms"] * 1e-3), paths_per_s=r["finite"] / (r["device_ms"] * 1e-3),
        track_ms=r["track_ms"], retrack_ms=r["escalate_ms"],
        finite=r["finite"], escalated=r["escalated"], oracle_checks=checks,
        form="one hc_track_batch, mixed precision")
    del b
    # ---- trifocal pose, unknown focal length
    fam = inputs.trifocal_family()
    z = np.load(os.path.join(START_DIR, "trifocal_f.npz"))
    gold = np.load(GOLDEN.replace("dense_sweep_oracle.json", "trifocal_oracle.npz"))
    I = args.trifocal_instances
    seeds = [int(sd) for sd in gold["scenes"]] + [30_000 + k for k in range(I - len(gold["scenes"]))]
    p1 = np.stack([inputs.trifocal_scene(sd)[0] for sd in seeds])
    pr = hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"],
                    symmetries=fam.sign_masks)
    t0 = time.perf_counter()
    b = pr.track(n_instances=I, p1=p1).wait()
    wall = time.perf_counter() - t0
    r = b.result
    c = gold["proj_coef"]
    checks = []
    for k in range(len(gold["scenes"])):
        ost = gold[f"status{k}"] & 0x7F
        gst = b.status[k] & 0x7F
        both = (ost == 1) & (gst == 1)
        gp, op = b.x[k][both] @ c, gold[f"proj{k}"][both]
        tol = np.sum(np.abs(c)) * 1e-8 * np.maximum(1.0, gold[f"xnorm{k}"][both])
        d, _ = cKDTree(np.stack([op.real, op.imag], 1)).query(np.stack([gp.real, gp.imag], 1))
        checks.append(dict(scene=seeds[k], status_diffs=int(np.sum(gst != ost)),
                           gpu_finite=int((gst == 1).sum()), oracle_finite=int((ost == 1).sum()),
                           finite_matched=int(np.sum(d <= tol))))
    out["trifocal_f"] = dict(
        instances=I, paths=r["paths"], device_ms=r["device_ms"], wall_ms=wall * 1e3,
        systems_per_s=I / (r["device_ms"] * 1e-3), paths_per_s=r["paths"] / (r["device_ms"] * 1e-3),
        track_ms=r["track_ms"], retrack_ms=r["escalate_ms"], finite=r["finite"],
        escalated=r["escalated"], golden_checks=checks,
        form="one hc_track_batch, mixed precision, one start per orbit of the quaternion signs")
    return out


# ---------------------------------------------------------------- batched solve (Fig. 3)
def solve_leg(hc, torch, stream, sizes=(4, 8, 12, 16, 20), batches=(1000, 100_000), reps=20):
    """The paper's Fig. 3 on this GPU: batches of n x n complex systems,
    hc_batched_solve (fused Gauss-Jordan in registers, one launch) against
    the library batched LU factorisation and solve as torch dispatches them
    (torch.linalg.lu_factor + lu_solve: cuBLAS / cuSOLVER / MAGMA batched
    routines, a black box here), FP32 and FP64 complex.  Times are CUDA-event
    means over `reps` calls on `stream`."""
    rows = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        ms = []
        for _ in range(reps + 2):
            ev0.record(stream)
            fn()
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return statistics.mean(ms[2:])

    for fp32 in (1, 0):
        dt = torch.complex64 if fp32 else torch.complex128
        esz = 8 if fp32 else 16
        for n in sizes:
            for batch in batches:
                g = torch.Generator(device="cuda").manual_seed(n * 7919 + batch)
                A = torch.randn((batch, n, n), dtype=dt, device="cuda", generator=g)
                b = torch.randn((batch, n), dtype=dt, device="cuda", generator=g)
                x = torch.empty_like(b)
                info = torch.empty(batch, dtype=torch.int32, device="cuda")
                out = {}
                with torch.cuda.stream(stream):
                    ours = timed(lambda: hc.batched_solve(A, b, x, info, stream.cuda_stream))

                    def lib():
                        LU, piv = torch.linalg.lu_factor(A)
                        out["x"] = torch.linalg.lu_solve(LU, piv, b.unsqueeze(-1))[..., 0]
                    ref = timed(lib)
                stream.synchronize()
                xr = out["x"]
                diff = float(((x - xr).abs().amax(dim=1) / xr.abs().amax(dim=1)).max())
                byt = batch * (n * n + 2 * n) * esz
                cfma = sum(j * (j + 1) for j in range(n)) + n * (n + 1) // 2
                rows.append(dict(dtype="c64" if fp32 else "c128", n=n, batch=batch,
                                 hc_us=ours * 1e3, library_us=ref * 1e3, speedup=ref / ours,
                                 hc_gbs=byt / (ours * 1e-3) / 1e9,
                                 hc_tflops=8.0 * cfma * batch / (ours * 1e-3) / 1e12,
                                 max_rel_diff_vs_library=diff, singular=int((info != 0).sum())))
    return dict(form="hc_batched_solve (one fused launch) vs torch.linalg.lu_factor + lu_solve "
                     "(library batched LU and triangular solves)", rows=rows)


# ---------------------------------------------------------------- CPU oracle
def class_sample(wl, total):
    """Paths per size class for a sample of `total` paths, proportional to the
    class's share of the step's paths (at least 4 each)."""
    P = [w["d"] ** w["n"] for w in wl]
    return [max(4, int(round(total * p / sum(P)))) for p in P]


def cpu_baseline(wl, bufs, args, sample=None, threads=None):
    """The FP64 oracle on a bounded sample: system 0 of each class, paths per
    class in proportion to the step; with bufs, its endpoints are compared
    with the GPU's of the same systems."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from hcmatch import match
    sample = sample or args.cpu_sample
    threads = threads or oracle.hardware_threads()
    t_total, n_paths = 0.0, 0
    worst, checked = 0.0, 0
    for si, (w, k) in enumerate(zip(wl, class_sample(wl, sample))):
        P = w["d"] ** w["n"]
        ids = np.random.default_rng(w["seeds"][0]).choice(P, size=min(k, P), replace=False)
        pr = oracle.OracleProblem(w["base"], gamma=w["gamma"], coef=w["coefs"][0])
        t0 = time.perf_counter()
        r = pr.track(path_ids=ids, threads=threads)
        t_total += time.perf_counter() - t0
        n_paths += len(ids)
        if bufs is not None:
            fin = (r["status"] & 0x7F) == oracle.FINITE
            _, dist = match(r["x"][fin], bufs[si]["x"][0], 1e-8)
            worst = max(worst, float(np.max(dist, initial=0.0)))
            checked += int(fin.sum())
    rate = n_paths / t_total
    return (dict(value=rate, unit="paths/s", cores=threads, kind="oracle",
                 sample=f"{n_paths} paths of system 0 of each size class, in proportion to "
                        f"the class's paths ({t_total:.1f} s)"),
            dict(checked=checked, max_rel_dist=worst, tol=1e-8, ok=worst <= 1e-8))


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: each step tracks a bounded
    sample of the workload (paths per class in proportion to the step) on all
    host cores."""
    rank, world = env_rank()
    if rank != 0:
        return None
    wl = workload(0)
    for _ in range(args.warmup):
        cpu_baseline(wl, None, args, sample=args.ref_sample)
    rates, cb = [], None
    for _ in range(args.steps):
        cb, _ = cpu_baseline(wl, None, args, sample=args.ref_sample)
        rates.append(cb["value"])
    value = statistics.median(rates)
    cb["value"] = value
    cb["sample"] = f"per step: {cb['sample']}"
    total_paths = sum(w["d"] ** w["n"] * SYSTEMS_PER_SIZE for w in wl)
    ms = total_paths / value * 1e3
    return dict(metric=METRIC, value=value, unit="paths/s", impl="reference", n_gpus=world,
                steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="c128", data="synthetic",
                config=dict(workload=WORKLOAD, paths_per_step=total_paths,
                            note="ms_per_step extrapolates the sampled rate to the full step"),
                cpu_baseline=cb,
                e2e=dict(value=value, unit="paths/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))


# ---------------------------------------------------------------- serving
def serving_problems(hc, precision, trifocal=True):
    """(name, problem, request generator) for the serving mix: dense
    quadratics n = 4..12, 4-view triangulation and trifocal pose."""
    probs = []
    for n in range(4, 13):
        probs.append((f"quad{n}", hc.Problem(inputs.dense_system(n, 2, 700 + n),
                                              gamma=inputs.unit_gamma(700 + n),
                                              settings=dict(precision=precision)),
                      lambda s, n=n: inputs.dense_coefficients(n, 2, s).reshape(-1)))
    z = np.load(os.path.join(START_DIR, "triangulation4.npz"))
    probs.append(("triangulation4", hc.Problem(inputs.triangulation_family(4).system,
                                                kind=hc.HC_PARAMETER, p0=z["p0"],
                                                start=z["start"],
                                                settings=dict(precision=precision)),
                  lambda s: inputs.triangulation_scene(s)[0]))
    if trifocal:
        z = np.load(os.path.join(START_DIR, "trifocal_f.npz"))
        fam = inputs.trifocal_family()
        probs.append(("trifocal_f", hc.Problem(fam.system, kind=hc.HC_PARAMETER, p0=z["p0"],
                                                start=z["start"], symmetries=fam.sign_masks,
                                                settings=dict(precision=precision)),
                      lambda s: inputs.trifocal_scene(s)[0]))
    return probs


def serve_run(hc, probs, rate, count, streams, max_batch, seed):
    """Poisson arrivals of `count` requests at `rate` per second, kinds
    uniform over probs; returns throughput and per-request latency."""
    rng = np.random.default_rng([seed, int(rate)])
    kinds = rng.integers(0, len(probs), size=count)
    gaps = rng.exponential(1.0 / rate, size=count)
    payload = [probs[k][2](10_000 + j) for j, k in enumerate(kinds)]
    srv = hc.Server(n_streams=streams, max_batch_instances=max_batch)
    ids = [None] * count
    t0 = time.perf_counter()

    def producer():
        t = t0
        for j, k in enumerate(kinds):
            t += gaps[j]
            while time.perf_counter() < t:
                pass
            ids[j] = srv.submit(probs[k][1], payload[j])

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    lat, paths, finite = [], 0, 0
    per_kind = {}
    for j, k in enumerate(kinds):
        x, st, info = srv.wait(ids[j], probs[k][1])
        lat.append(info["latency_us"] / 1e3)
        paths += info["paths"]
        finite += info["finite"]
        per_kind.setdefault(probs[k][0], []).append(info["latency_us"] / 1e3)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    return dict(offered_per_s=rate, requests=count, systems_per_s=count / wall,
                paths_per_s=finite / wall, p50_ms=float(np.percentile(lat, 50)),
                p99_ms=float(np.percentile(lat, 99)), recovery=finite / paths,
                batches=stats["batches"], max_inflight_batches=stats["max_inflight_batches"],
                p50_ms_by_kind={k: float(np.percentile(v, 50)) for k, v in sorted(per_kind.items())})


def stream_run(hc, problem, gen, rate, count, slots, seed, cap_s=20.0):
    """Poisson arrivals of `count` requests of one kind at `rate` per second
    into a resident launch (hc.Stream, continuous admission): one host
    thread submits each request at its arrival time and collects finished
    ones in between; latency = arrival to collection.  Stops after cap_s
    (the requests collected by then are reported)."""
    rng = np.random.default_rng([seed, int(rate), 7])
    arrive = np.cumsum(rng.exponential(1.0 / rate, size=count))
    payload = [gen(20_000 + j) for j in range(count)]
    st = hc.Stream(problem, slots=slots, idle_us=20000)
    kind = problem.kind
    pending, lat, paths, finite = [], [], 0, 0
    j = 0
    t0 = time.perf_counter()
    while (j < count or pending) and time.perf_counter() - t0 < cap_s:
        now = time.perf_counter() - t0
        if j < count and now >= arrive[j]:
            try:
                tk = st.submit(p1=payload[j]) if kind != hc.HC_TOTAL_DEGREE else \
                    st.submit(coef=payload[j])
                pending.append((j, tk))
                j += 1
                continue
            except hc.HCError:  # every slot in use: collect below
                pass
        if pending:
            jj, tk = pending[0]
            r = st.poll(tk, timeout_us=0 if j < count else 200)
            if r is not None:
                pending.pop(0)
                lat.append((time.perf_counter() - t0 - arrive[jj]) * 1e3)
                paths += len(r[1])
                finite += int(np.sum((r[1] & 0x7F) == hc.PATH_FINITE))
                continue
        if j < count:
            time.sleep(max(0.0, min(50e-6, arrive[j] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    st.close()
    done = len(lat)
    return dict(offered_per_s=rate, requests=count, completed=done, systems_per_s=done / wall,
                paths_per_s=finite / wall, p50_ms=float(np.percentile(lat, 50)) if lat else None,
                p99_ms=float(np.percentile(lat, 99)) if lat else None,
                recovery=finite / paths if paths else None)


def stream_rows(hc, rates, duration):
    """Continuous admission against the batch server on single-kind Poisson
    streams: dense quadratics n = 8 (256 paths per request, almost no
    re-tracking) at the given rates, and 4-view triangulation (296 paths, a
    quarter of them re-tracked) at the lowest rate."""
    z = np.load(os.path.join(START_DIR, "triangulation4.npz"))
    kinds = [("triangulation4", hc.Problem(inputs.triangulation_family(4).system,
                                           kind=hc.HC_PARAMETER, p0=z["p0"], start=z["start"]),
              lambda s: inputs.triangulation_scene(s)[0]),
             ("quad8", hc.Problem(inputs.dense_system(8, 2, 708), gamma=inputs.unit_gamma(708)),
              lambda s: inputs.dense_coefficients(8, 2, s).reshape(-1))]
    rows = []
    for name, pr, gen in kinds[::-1]:
        for rate in (rates if name == "quad8" else rates[:1]):
            count = int(max(50, min(rate * duration, 20000)))
            rows.append(dict(kind=name, form="resident launch (hc_stream)",
                             **stream_run(hc, pr, gen, rate, count, 256, 3)))
            rows.append(dict(kind=name, form="batch server (hc_server)",
                             **{k: v for k, v in serve_run(hc, [(name, pr, gen)], rate, count, 4,
                                                           64, 3).items()
                                if k not in ("batches", "max_inflight_batches",
                                             "p50_ms_by_kind")}))
    return rows


def serve_rows(hc, rates, duration, trifocal=True, fp64_requests=0):
    mixed = serving_problems(hc, hc.HC_PREC_MIXED, trifocal)
    rows = []
    for rate in rates:
        count = int(max(50, min(rate * duration, 20000)))
        rows.append(dict(form="mixed continuous batching", kinds=[p[0] for p in mixed],
                         **serve_run(hc, mixed, rate, count, 4, 64, 1)))
    if fp64_requests:
        fp64 = serving_problems(hc, hc.HC_PREC_FP64, trifocal)
        rows.append(dict(form="plain FP64, one launch per system",
                         **serve_run(hc, fp64, rates[0], fp64_requests, 1, 1, 1)))
    return rows


def serve_mix(args):
    """Serving sweep: Poisson arrivals at several rates, continuous batching
    on the GPU versus the plain FP64 one-launch-per-system form."""
    import torch
    from paper_2112_03444_gb300 import hc
    torch.cuda.set_device(0)
    rows = serve_rows(hc, [float(r) for r in args.rates.split(",")], args.duration,
                      trifocal=not args.no_trifocal, fp64_requests=args.fp64_requests)
    print(json.dumps(dict(metric=METRIC, mode="serving", rows=rows)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=320,
                    help="oracle paths (all host cores) for cpu_baseline")
    ap.add_argument("--cpu-sample-1t", type=int, default=40,
                    help="oracle paths (one thread) for cpu_baseline_1thread")
    ap.add_argument("--ref-sample", type=int, default=160,
                    help="oracle paths per step of the reference arm")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--no-serving-leg", action="store_true")
    ap.add_argument("--no-solve-leg", action="store_true")
    ap.add_argument("--no-param-legs", action="store_true")
    ap.add_argument("--no-admission-leg", action="store_true")
    ap.add_argument("--admission-rates", default="400,2000,8000")
    ap.add_argument("--admission-duration", type=float, default=1.0)
    ap.add_argument("--tri-instances", type=int, default=10_000)
    ap.add_argument("--trifocal-instances", type=int, default=1000)
    ap.add_argument("--serve-rate", type=float, default=400.0,
                    help="offered requests/s of the serving leg")
    ap.add_argument("--serve-duration", type=float, default=2.0)
    ap.add_argument("--serve", action="store_true",
                    help="serving sweep: Poisson arrivals, continuous batching vs plain FP64")
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000")
    ap.add_argument("--duration", type=float, default=2.0)
    ap.add_argument("--fp64-requests", type=int, default=60)
    ap.add_argument("--no-trifocal", action="store_true")
    args = ap.parse_args()
    if args.serve:
        serve_mix(args)
        return
    if args.impl == "reference":
        line = run_reference(args)
    else:
        line = run_gpu(args)
    rank, _ = env_rank()
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

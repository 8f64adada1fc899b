"""Benchmark: batched homotopy-continuation path tracking on one GB300.

Workload (dense total-degree sweep): dense random quadratic systems with
n = 8, 10, 12 unknowns (256 / 1024 / 4096 paths each) and dense random cubic
systems with n = 6, 8 (729 / 6561 paths), complex Gaussian coefficients,
16 systems per size; every path of every system of a size runs in one
persistent mixed-precision launch (FP32 tracking, FP64 endgame residuals and
refinement).  One step = all five size classes, 202,656 paths.

Prints one JSON line: value = matched paths/s (paths whose endpoint is a
finite root; the Bezout count d^n is checked for every system, and a sampled
set of FP64 oracle endpoints must be found among the GPU's within 1e-8).
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

SIZES = [(8, 2), (10, 2), (12, 2), (6, 3), (8, 3)]   # (n, degree)
SYSTEMS_PER_SIZE = 16
SEED0 = 100
WORKLOAD = "dense total-degree sweep: quadratics n=8,10,12; cubics n=6,8; 16 systems per size"
METRIC = "paths/s and systems/s at oracle-matched roots (1e-8); p50/p99 latency per system"
FP32_LANES_PER_SM = 128
SM_COUNT = 152


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


def workload(rank=0):
    """Per size: (n, d, base TermSystem, coefficient array [16, T], gamma)."""
    from paper_2112_03444_gb300 import inputs
    out = []
    for si, (n, d) in enumerate(SIZES):
        seeds = [SEED0 + 1000 * rank + 100 * si + k for k in range(SYSTEMS_PER_SIZE)]
        base, coefs = inputs.dense_batch(n, d, seeds)
        out.append(dict(n=n, d=d, base=base, coefs=coefs, seeds=seeds,
                        gamma=inputs.unit_gamma(seeds[0])))
    return out


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
    f = dense_flops_per_unit(n, d)
    rk = 4 * (f["E_Hx"] + f["E_Ht"] + f["S"])
    nw = f["E_H"] + f["E_Hx"] + f["S"]
    return 8.0 * (steps * rk + newton * nw)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
    # one stream per size class: the five persistent launches (and their FP64
    # re-tracking launches) overlap on the device
    class_streams = [torch.cuda.Stream(device=dev) for _ in SIZES]
    wl = workload(rank)
    settings = dict(precision=hc.HC_PREC_MIXED)
    problems, bufs = [], []
    for w in wl:
        pr = hc.Problem(w["base"], gamma=w["gamma"], settings=settings)
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
            pr, b, cs = problems[i], bufs[i], class_streams[i]
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

    # ---- correctness of the measured run: Bezout count per system
    last = results[-1]
    finite = 0
    for w, b in zip(wl, bufs):
        st = b["st"].cpu().numpy() & 0x7F
        per = (st == hc.PATH_FINITE).sum(axis=1)
        finite += int(per.sum())
    recovery = finite / total_paths

    # ---- dominant kernel roofline: the tracking launch of the class with the
    # most algorithmic work in the timed step (from its device step
    # counters), timed alone (inside the step the five classes overlap, so a
    # launch's wall time there includes waiting for SM slots)
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
        # flops of the tracking launch only: all steps minus the FP64 tier's
        dflop.append(flops(dw["n"], dw["d"],
                           r["steps_accepted"] + r["steps_rejected"] - r["esc_accepted"] - r["esc_rejected"],
                           r["newton_iters"] - r["esc_newton"]))
        bt.close()
    achieved = statistics.mean(f / (m * 1e-3) for f, m in zip(dflop, dk_ms)) / 1e12
    peak_fp32, _ = hc.measure_fma_peak(False)
    peak = peak_fp32 / 1e12

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

    # ---- the same sweep as one launch per system (mixed tiers, one stream):
    # the form the batched persistent launches replace
    per_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        bts = []
        for i in order:
            pr, b = problems[i], bufs[i]
            for k in range(SYSTEMS_PER_SIZE):
                bts.append(pr.track(n_instances=1, coef=b["coef"][k:k + 1], device=True,
                                    x_out=b["x"][k:k + 1], status_out=b["st"][k:k + 1],
                                    steps_out=b["steps"][k:k + 1], be_out=b["be"][k:k + 1],
                                    stream=sp))
        s1.record(stream)
        for bt in bts:
            bt.wait()
        torch.cuda.synchronize()
        per_ms.append(s0.elapsed_time(s1))
        for bt in bts:
            bt.close()
    per_system = dict(value=total_paths * recovery * world / (min(per_ms) * 1e-3), unit="paths/s",
                      ms_per_step=min(per_ms),
                      form="one hc_track_batch per system, mixed tiers, one stream, device buffers")

    line = dict(
        metric=METRIC, value=total_paths * recovery * world / (ms * 1e-3), unit="paths/s",
        systems_per_s=total_systems * world / (ms * 1e-3),
        latency_ms=dict(p50=statistics.median(step_ms), p99=float(np.percentile(step_ms, 99)),
                        note="whole-batch latency per system (all systems of a step finish together)"),
        n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="c64+c128 (mixed)",
        data="synthetic",
        config=dict(workload=WORKLOAD, paths_per_step=total_paths, systems_per_step=total_systems,
                    precision="mixed FP32 tracking, FP64 endgame/refinement",
                    l2="flushed between timed steps (256 MB write)", parallelism=f"replicas{world}",
                    launch="one captured CUDA graph per size class (hc_plan_run), five streams"),
        recovery=recovery,
        escalated=sum(r["escalated"] for r in last),
        e2e=dict(value=total_paths * recovery * world / (e2e * 1e-3), unit="paths/s",
                 h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, ms_per_step=e2e,
                 path="hc_plan_run per size class on its own stream, pinned host buffers",
                 same_statuses_as_device_run=e2e_ok),
        gpu_launches=launches,
        one_system_per_launch=per_system,
        roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                      frac=achieved / peak, traffic=recorded_traffic(),
                      kernel=f"dense_td_kernel<n={dw['n']}, d={dw['d']}, mixed>",
                      kernel_ms=statistics.mean(dk_ms),
                      peak_note="of measured: FP32 FMA throughput from hc_measure_fma_peak on this "
                                "GPU in this run; algorithmic flops from the device step counters"),
        clocks=clocks,
    )
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"], match = cpu_baseline(wl, bufs, args)
        line["oracle_match"] = match
    if world > 1:
        dist.destroy_process_group()
    return line


# ---------------------------------------------------------------- CPU oracle
def cpu_baseline(wl, bufs, args, sample=None):
    """Oracle on a bounded sample: paths per size class from system 0."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from hcmatch import match
    sample = sample or args.cpu_sample
    threads = oracle.hardware_threads()
    t_total, n_paths = 0.0, 0
    worst, checked = 0.0, 0
    for si, w in enumerate(wl):
        P = w["d"] ** w["n"]
        ids = np.random.default_rng(w["seeds"][0]).choice(P, size=min(sample, P), replace=False)
        pr = oracle.OracleProblem(w["base"], gamma=w["gamma"], coef=w["coefs"][0])
        t0 = time.perf_counter()
        r = pr.track(path_ids=ids, threads=threads)
        t_total += time.perf_counter() - t0
        n_paths += len(ids)
        if bufs is not None:
            gx = bufs[si]["x"][0].cpu().numpy()
            _, dist = match(r["x"], gx, 1e-8)
            worst = max(worst, float(np.max(dist)))
            checked += len(ids)
    rate = n_paths / t_total
    return (dict(value=rate, unit="paths/s", cores=threads, kind="oracle",
                 sample=f"{sample} paths per size class (system 0 of each), {n_paths} paths, "
                        f"{t_total:.1f} s"),
            dict(checked=checked, max_rel_dist=worst, tol=1e-8, ok=worst <= 1e-8))


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: each step tracks a bounded
    sample of the workload (ref_sample paths per size class) on all host cores."""
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
def serve_mix(args):
    """Poisson arrivals of single-system requests drawn from {dense quadratics
    n = 4..12, 4-view triangulation, trifocal pose}: continuous batching on
    the GPU versus the plain FP64 one-launch-per-system form."""
    import threading
    import torch
    from paper_2112_03444_gb300 import hc, inputs
    torch.cuda.set_device(0)
    start_dir = os.path.join(ROOT, "paper_2112_03444_gb300", "startsets")

    def problems(precision):
        probs = []
        for n in range(4, 13):
            probs.append((f"quad{n}", hc.Problem(inputs.dense_system(n, 2, 700 + n),
                                                  gamma=inputs.unit_gamma(700 + n),
                                                  settings=dict(precision=precision)),
                          lambda s, n=n: inputs.dense_coefficients(n, 2, s).reshape(-1)))
        z = np.load(os.path.join(start_dir, "triangulation4.npz"))
        probs.append(("triangulation4", hc.Problem(inputs.triangulation_family(4).system,
                                                    kind=hc.HC_PARAMETER, p0=z["p0"],
                                                    start=z["start"],
                                                    settings=dict(precision=precision)),
                      lambda s: inputs.triangulation_scene(s)[0]))
        tf = os.path.join(start_dir, "trifocal_f.npz")
        if os.path.exists(tf) and not args.no_trifocal:
            z = np.load(tf)
            probs.append(("trifocal_f", hc.Problem(inputs.trifocal_family().system,
                                                    kind=hc.HC_PARAMETER, p0=z["p0"],
                                                    start=z["start"],
                                                    settings=dict(precision=precision)),
                          lambda s: inputs.trifocal_scene(s)[0]))
        return probs

    def run(probs, rate, count, streams, max_batch, seed):
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
        for j, k in enumerate(kinds):
            x, st, info = srv.wait(ids[j], probs[k][1])
            lat.append(info["latency_us"] / 1e3)
            paths += info["paths"]
            finite += info["finite"]
        wall = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        return dict(offered_per_s=rate, requests=count, systems_per_s=count / wall,
                    paths_per_s=finite / wall, p50_ms=float(np.percentile(lat, 50)),
                    p99_ms=float(np.percentile(lat, 99)), recovery=finite / paths,
                    batches=stats["batches"], max_inflight_batches=stats["max_inflight_batches"])

    mixed = problems(hc.HC_PREC_MIXED)
    rows = []
    for rate in [float(r) for r in args.rates.split(",")]:
        count = int(max(50, min(rate * args.duration, 20000)))
        rows.append(dict(form="mixed continuous batching", **run(mixed, rate, count, 4, 64, 1)))
    fp64 = problems(hc.HC_PREC_FP64)
    rate = float(args.rates.split(",")[0])
    rows.append(dict(form="plain FP64, one launch per system",
                     **run(fp64, rate, args.fp64_requests, 1, 1, 1)))
    line = dict(metric=METRIC, mode="serving", workload="Poisson mix of " +
                ", ".join(p[0] for p in mixed), rows=rows)
    print(json.dumps(line), flush=True)


def run_case(spec):
    """One dense size class, tracked twice (for profilers): spec = "n,d,instances"."""
    import torch
    from paper_2112_03444_gb300 import hc, inputs
    n, d, ni = (int(v) for v in spec.split(","))
    torch.cuda.set_device(0)
    seeds = [SEED0 + k for k in range(ni)]
    base, coefs = inputs.dense_batch(n, d, seeds)
    pr = hc.Problem(base, gamma=inputs.unit_gamma(seeds[0]), settings=dict(escalate=0))
    for _ in range(2):
        bt = pr.track(n_instances=ni, coef=coefs).wait()
    print(json.dumps(dict(case=spec, **bt.result)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=160)
    ap.add_argument("--ref-sample", type=int, default=48)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="serving mix: Poisson arrivals, continuous batching vs plain FP64")
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000")
    ap.add_argument("--duration", type=float, default=2.0)
    ap.add_argument("--fp64-requests", type=int, default=60)
    ap.add_argument("--no-trifocal", action="store_true")
    ap.add_argument("--case", default=None,
                    help="profiling helper: track one dense class 'n,d,instances' twice and exit")
    args = ap.parse_args()
    if args.case:
        run_case(args.case)
        return
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

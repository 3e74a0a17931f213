#!/usr/bin/env python
"""Benchmark: spin-flip attempts per second of parallel-tempering Metropolis on the 2D
Ising model, batched path vs the plain one-problem-per-launch path, on B300, plus the
continuous-batching server's p50/p99 latency.

Default workload (one step): 256 independent PT problems, L uniform over
{32, 48, 64, 96, 128, 256}, R uniform in 8..48, betas linear 0.30 -> 0.60, J = 1, h = 0,
2000 sweeps each with an exchange after every sweep, advanced by one pt_sweep_batch call.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|single|serve|flip|converge] [--field H]
                    [--streams S] [--quick]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank runs its own copy of the
workload on its own GPU (independent problems, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/sec (all replicas, 1 B300) batched vs plain; serve p50/p99"
UNIT = "attempts/s"
MUL_PER_ATTEMPT = 5.0  # Philox4x32-10: 20 32x32->64 products per block of 4 draws
IMUL_WIDE_PER_CLK_SM = 32.0  # 32x32->64 integer products per clock per SM (4 SMSPs x 8)
# The issue bound of the roofline: about 25 integer operations per attempt (a quarter of a
# Philox4x32-10 block of ~78 operations, plus ~5 for the update: class masks, threshold
# compare, flip insert and a share of the bit-sliced neighbour count), against 4 schedulers x
# 32 lanes issuing one operation per clock on every SM.
OPS_PER_ATTEMPT = 25.0
LANE_OPS_PER_CLK_SM = 128.0

# DRAM traffic of one k_flat_half launch (colour 0) on the batched-256 workload, from an ncu
# capture of that launch (dram__bytes_read.sum + dram__bytes_write.sum; cold caches: one read
# of the whole state). Valid only for the kernel source it was taken on.
FLAT_TRAFFIC_BYTES = 25.978368e6 + 0.0
FLAT_TRAFFIC_SOURCES = ("paper_2512_03825_b300/csrc/pt_device.cuh",
                        "paper_2512_03825_b300/csrc/pt_flat.cuh",
                        "paper_2512_03825_b300/csrc/pt_flat.cu")
FLAT_TRAFFIC_SOURCE_HASH = "21eb1116c7d57edf"


def _flat_traffic():
    import hashlib
    h = hashlib.sha256()
    for rel in FLAT_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return FLAT_TRAFFIC_BYTES if h.hexdigest()[:16] == FLAT_TRAFFIC_SOURCE_HASH else None


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["batched", "single", "serve", "flip", "converge"],
                    default="batched")
    ap.add_argument("--sizes", type=str, default="16,32,64,128,256",
                    help="lattice sizes of --workload converge")
    ap.add_argument("--seeds", type=int, default=8, help="seeds per size of --workload converge")
    ap.add_argument("--iterations", type=int, default=300_000,
                    help="single-spin-flip iterations per replica per step (--workload flip)")
    ap.add_argument("--sweeps", type=int, default=2000, help="sweeps per problem per step")
    ap.add_argument("--problems", type=int, default=256)
    ap.add_argument("--field", type=float, default=0.0,
                    help="field h of the batched workload's problems (J = 1; h != 0 runs the "
                         "generic update)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving leg of the default line")
    ap.add_argument("--requests", type=int, default=2000,
                    help="requests of --workload serve")
    ap.add_argument("--sweep-strategy", choices=["auto", "launches", "persistent", "bands"],
                    default="auto", help="plain-path strategy of --workload single (auto: the "
                                         "tuned shape of the problem, else the library's "
                                         "default)")
    ap.add_argument("--single", choices=["L16_R8", "L128_R32", "L1024_R64"],
                    default="L1024_R64", help="the problem of --workload single")
    ap.add_argument("--streams", type=int, default=None,
                    help="streams of the lock-step batch (default: the tuned choice)")
    ap.add_argument("--graphs", type=int, choices=[0, 1], default=None,
                    help="graph replay of the lock-step batch (default: the tuned choice)")
    ap.add_argument("--quick", action="store_true",
                    help="skip the side measurements (plain path, L1024, e2e, CPU baseline)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------------
# distributed plumbing (one process per GPU; weak scaling over independent problems)
# ---------------------------------------------------------------------------------------
def dist_setup(args, backend="nccl"):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    """The slowest rank's value (timing): the job is done when every rank is."""
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX if world > 1 else None)


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM if world > 1 else None)


RANK_SEED_STRIDE = 0x10000


def rank_problems(rank, n, sweeps, every=1, h=0.0):
    """This rank's share of the work: its own copy of the batched workload with seeds offset
    by rank, so every rank advances different (independent) problems of the same shape; h is
    the problems' field."""
    from paper_2512_03825_b300 import workloads as W
    import dataclasses
    probs = W.batched_problems(n=n, sweeps=sweeps, every=every)
    return [dataclasses.replace(p, seed=p.seed + rank * RANK_SEED_STRIDE, h=h) for p in probs]


def job_throughput(attempts_this_rank, seconds_this_rank, world):
    """Whole-job attempts per second: all ranks' attempts over the slowest rank's time."""
    total = sum_over_ranks(attempts_this_rank, world)
    slowest = max_over_ranks(seconds_this_rank, world)
    return total / slowest, total, slowest


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def batched_config(args, per_step):
    """The `config` of the batched workload's line: the same dict in both arms."""
    return {
        "workload": "batched-256: %d PT problems, L in {32,48,64,96,128,256}, R 8-48, "
                    "betas 0.30-0.60, J=1, h=%g, %d sweeps, exchange every sweep"
                    % (args.problems, args.field, args.sweeps),
        "problems": args.problems, "sweeps_per_step": args.sweeps, "exchange_every": 1,
        "attempts_per_step": per_step, "parallelism": "independent problems per GPU",
        "l2": "flushed (256 MiB write) between timed steps",
    }


def _attempts(probs, sweeps):
    return float(sum(p.L * p.L * p.R for p in probs)) * sweeps


def run_ours(args, rank, world, local):
    import torch

    from paper_2512_03825_b300 import api
    from paper_2512_03825_b300 import workloads as W
    from paper_2512_03825_b300 import autotune

    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    api.use_torch_allocator(True)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    tuning = autotune.apply_cached_or_default()
    if args.streams is not None:
        tuning = dict(tuning, streams=args.streams)
        autotune.set_tuning(**tuning)
    if args.graphs is not None:
        tuning = dict(tuning, graphs=args.graphs)
        autotune.set_tuning(**tuning)

    if args.workload == "single":
        return run_single(args, rank, world, stream, sms)
    if args.workload == "flip":
        return run_flip(args, rank, world, stream)
    if args.workload == "converge":
        return run_converge(args, rank, world, stream)
    if args.workload == "serve":
        from paper_2512_03825_b300 import serve
        res = serve.bench_serve(args, rank, world, stream)
        return {"metric": METRIC, "value": res["attempts_per_s"], "unit": UNIT,
                "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * res["wall_s"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic Poisson request stream",
                "config": {"workload": "serving: %d Poisson PT requests, L 32-512, R 8-64, "
                                       "sweeps 1e2-1e4, h in {0, 0.1}, 80 GB budget"
                                       % args.requests},
                "serve": res}

    probs = rank_problems(rank, args.problems, args.sweeps, 1, args.field)
    handles = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=stream)
               for p in probs]
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    per_step = _attempts(probs, args.sweeps)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            api.sweep_batch(handles, args.sweeps, 1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(dev)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()                     # evict the lattices from L2 between steps
            ev[k][0].record(stream)
            api.sweep_batch(handles, args.sweeps, 1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - t0
        clk = clocks.stop()
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    value, _, total_s = job_throughput(per_step * args.steps, sum(kernel_ms) / 1e3, world)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded problem mix; random +-1 initial spins)",
        "config": batched_config(args, per_step),
        "batch_tuning": tuning,
        "clocks": clk,
        "gpu_launches": args.steps * launches_per_batch(probs, args.sweeps, tuning),
        "wall_s": wall,
    }
    peaks = measured_peaks()
    clock_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    peak_mul = sms * IMUL_WIDE_PER_CLK_SM * clock_mhz * 1e6
    peak_ops = sms * LANE_OPS_PER_CLK_SM * clock_mhz * 1e6
    flat = tuning.get("strategy", 0) in (0, 3)  # lock-step: dealt or queued tiles
    overlapped = None
    if flat:
        # the dominant kernel on its own: a batch without exchanges is nothing but
        # k_flat_half launches (two per sweep), timed on the problems' stream. Two batch
        # lengths, so that the per-call host work (tile dealing, list upload) cancels in
        # the difference. First on one stream (one launch per half sweep covers every
        # problem: the kernel's own launch duration), then in the tuned number of parts on
        # their own streams (their launches overlap: the effective time per half sweep).
        lens = (100, 500)

        def half_sweep_s(streams):
            autotune.set_tuning(**dict(tuning, streams=streams))
            took = []
            with torch.cuda.stream(stream):
                for nsw in lens:
                    # one untimed call of the same shape first (with graph replay on, it is
                    # the call that captures)
                    api.sweep_batch(handles, nsw, 0)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    api.sweep_batch(handles, nsw, 0)
                    b.record(stream)
                    torch.cuda.synchronize()
                    took.append(a.elapsed_time(b) / 1e3)
            autotune.set_tuning(**tuning)
            return (took[1] - took[0]) / (2 * (lens[1] - lens[0]))

        launch_s = half_sweep_s(1)
        att_per_s = per_step / args.sweeps / 2 / launch_s
        how = ("k_flat_half: attempts of one half sweep of all %d problems (one launch on one "
               "stream) / its average launch duration, (t(%d sweeps) - t(%d sweeps)) / %d "
               "launches (CUDA events on the problems' stream)"
               % (len(probs), lens[1], lens[0], 2 * (lens[1] - lens[0])))
        traffic = _flat_traffic() if args.field == 0.0 else None
        if tuning.get("streams", 1) > 1:
            ov = per_step / args.sweeps / 2 / half_sweep_s(tuning["streams"])
            overlapped = {"streams": tuning["streams"],
                          "achieved": OPS_PER_ATTEMPT * ov / 1e12,
                          "frac": OPS_PER_ATTEMPT * ov / peak_ops,
                          "note": "the same half sweeps with the batch in %d parts on their own "
                                  "streams (the tuned shape): their launches overlap, so this "
                                  "is the effective rate, not one launch's"
                                  % tuning["streams"]}
    else:
        att_per_s = per_step / (statistics.mean(kernel_ms) / 1e3)
        how = "k_batch: attempts of one batch / its duration"
        traffic = None
    step_att_per_s = value / world
    out["roofline"] = {
        "bound": "alu",
        "kernel": "k_flat_half" if flat else "k_batch",
        "achieved": OPS_PER_ATTEMPT * att_per_s / 1e12, "peak": peak_ops / 1e12,
        "unit": "T int-ops/s", "frac": OPS_PER_ATTEMPT * att_per_s / peak_ops,
        "traffic": traffic,
        "step_frac": OPS_PER_ATTEMPT * step_att_per_s / peak_ops,
        "overlapped": overlapped,
        "mul_pipe": {"achieved": MUL_PER_ATTEMPT * att_per_s / 1e12,
                     "peak": peak_mul / 1e12, "unit": "T int-mul/s",
                     "frac": MUL_PER_ATTEMPT * att_per_s / peak_mul,
                     "step_frac": MUL_PER_ATTEMPT * step_att_per_s / peak_mul},
        "note": "issue bound: %d integer operations per attempt (analytic: a quarter Philox4x32-10 "
                "block plus the update) against %d SMs x %d lane-operations per clock x %.0f MHz "
                "(max clock; measured SM count); %s; step_frac = the whole timed step (both half "
                "sweeps, the bond count and the exchange launch) on the same bound; mul_pipe = "
                "the same attempts as 32x32->64 products (5 per attempt) against %d per clock "
                "per SM, the higher of the two ceilings; traffic = DRAM bytes per launch from ncu "
                "(cold caches)" % (OPS_PER_ATTEMPT, sms, LANE_OPS_PER_CLK_SM, clock_mhz, how,
                                   IMUL_WIDE_PER_CLK_SM),
    }
    if not args.quick and rank == 0:
        out["serve"] = bench_serve_short(stream, args.serve_requests)
        if args.field == 0.0:
            out["batched_h0.1"] = bench_batched_variant(stream, args.problems, args.sweeps, 0.1)
            # sixteen times the problems: the spin words alone (about 360 MB) exceed the L2
            out["batched_4096"] = bench_batched_variant(stream, 16 * args.problems, 100, 0.0)
        out["plain"] = bench_plain(probs, args.sweeps, stream)
        out["batched_vs_plain"] = value / world / out["plain"]["value"]
        out["single_L1024_R64"] = bench_single(stream, sms, clock_mhz)
        out["single_L128_R32"] = bench_single(stream, sms, clock_mhz, "L128_R32", 2000)
        out["single_L16_R8"] = bench_single(stream, sms, clock_mhz, "L16_R8", 1000)
        from paper_2512_03825_b300 import workloads as W
        out["paper_L300_R1500"] = bench_single(stream, sms, clock_mhz, sweeps=300,
                                               prob=W.paper_problem())
        out["paper_single_flip_full_run"] = bench_paper_flip(stream)
        out["e2e"] = bench_e2e(probs, args.sweeps, stream, world, args.steps)
        out["cpu_baseline"] = cpu_baseline_plan(probs)
    elif not args.quick:
        bench_e2e(probs, args.sweeps, stream, world, args.steps)
    for h in handles:
        h.close()
    return out


def launches_per_batch(probs, sweeps, tuning):
    """Kernel launches of one pt_sweep_batch call: the lock-step strategies (dealt or queued
    tiles) launch, for each part of the batch (one per stream), two half sweeps per sweep
    plus one exchange launch after every sweep with an exchange (one mode here: h = 0); the
    dataflow strategy is one cooperative launch per mode; the cluster strategy is one
    persistent launch plus a helper."""
    strategy = tuning.get("strategy", 0)
    if strategy in (0, 3):  # per sweep and part of the batch (one part per stream)
        return sweeps * 3 * max(1, min(tuning.get("streams", 1), len(probs)))
    if strategy == 2:
        return len({p.h == 0.0 and p.J > 0 for p in probs})
    return 2


def bench_serve_short(stream, nreq):
    """The serving workload: `nreq` Poisson requests (default 2000, the whole stream) at 80%
    of the measured batched rate, an 80 GB budget."""
    from paper_2512_03825_b300 import serve

    class A:
        requests = nreq
    out = serve.bench_serve(A, 0, 1, stream)
    out["note"] = "%d Poisson requests at 80%% of the measured batched rate" % nreq
    return out


def _plain_run(sample, sweeps, strategy, stream):
    import torch
    from paper_2512_03825_b300 import api
    hs = [api.PTProblem(p.L, p.betas, seed=p.seed, stream=stream) for p in sample]
    for h in hs:
        h.set_sweep_tuning(strategy)
        h.sweep(5, 1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for h in hs:
        h.sweep(sweeps, 1)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    for h in hs:
        h.close()
    return _attempts(sample, sweeps) / (ms / 1e3)


def bench_batched_variant(stream, n, sweeps, h, steps=2):
    """The default step's problem mix, n problems with a field h (J = 1; h != 0 runs the
    generic update: five threshold classes with dE > 0 for 0 < h < 2), the same batch call,
    `steps` timed batches of `sweeps` sweeps with an exchange after every sweep, L2 flushed
    between them."""
    import torch
    from paper_2512_03825_b300 import api
    probs = rank_problems(0, n, sweeps, 1, h)
    hs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=stream) for p in probs]
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    took = []
    with torch.cuda.stream(stream):
        api.sweep_batch(hs, sweeps, 1)  # untimed, the same shape as the timed calls
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            api.sweep_batch(hs, sweeps, 1)
            b.record(stream)
            torch.cuda.synchronize()
            took.append(a.elapsed_time(b) / 1e3)
    for g in hs:
        g.close()
    t = statistics.mean(took)
    spin_bytes = sum(p.L * p.L * ((p.R + 31) // 32) * 4 for p in probs)
    return {"value": _attempts(probs, sweeps) / t, "unit": UNIT, "h": h, "problems": n,
            "sweeps": sweeps, "every": 1, "steps": steps, "us_per_sweep": 1e6 * t / sweeps,
            "spin_state_mb": spin_bytes / 1e6}


def bench_plain(probs, sweeps, stream, n_sample=32, sample_sweeps=200):
    """The plain path -- one problem at a time through pt_sweep -- on the same workload: every
    problem for the same number of sweeps with its default strategy (one persistent launch
    per call); the other strategy (one launch per half sweep plus the exchange launches),
    about 2.5x slower, on a sample of the same mix (every 8th problem, 200 sweeps)."""
    full = _plain_run(probs, sweeps, 2, stream)
    sample = probs[:: max(1, len(probs) // n_sample)][:n_sample]
    launches = _plain_run(sample, sample_sweeps, 1, stream)
    return {"value": full, "unit": UNIT, "problems": len(probs), "sweeps": sweeps,
            "launches": len(probs), "strategy": "persistent (one launch per problem)",
            "launches_strategy": {"value": launches, "problems": len(sample),
                                  "sweeps": sample_sweeps,
                                  "launches": len(sample) * sample_sweeps * 4}}


def bench_single(stream, sms, clock_mhz, name="L1024_R64", sweeps=200, prob=None):
    """One single-problem config on the plain path (pt_sweep), in the shape the plain-path
    autotuner cached for it on this device, else the library's default strategy."""
    import torch
    from paper_2512_03825_b300 import api, autotune
    from paper_2512_03825_b300 import workloads as W
    p = prob if prob is not None else W.SINGLE[name]
    h = api.PTProblem(p.L, p.betas, seed=p.seed, stream=stream)
    tuned = autotune.apply_single(h, p.L, p.R, p.J, p.h)
    h.sweep(10, p.every)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    h.sweep(sweeps, p.every)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    strategy, wpt, grid = h.sweep_tuning()
    h.close()
    att = float(p.L * p.L * p.R * sweeps)
    v = att / (ms / 1e3)
    peak_att = sms * IMUL_WIDE_PER_CLK_SM * clock_mhz * 1e6 / MUL_PER_ATTEMPT
    peak_issue = sms * LANE_OPS_PER_CLK_SM * clock_mhz * 1e6 / OPS_PER_ATTEMPT
    return {"value": v, "unit": UNIT, "sweeps": sweeps, "every": p.every,
            "frac_of_issue_roofline": v / peak_issue,
            "frac_of_mul_roofline": v / peak_att, "us_per_sweep": 1e3 * ms / sweeps,
            "sweep_strategy": strategy, "words_per_thread": wpt, "persistent_grid": grid,
            "tuned": tuned is not None}


def bench_paper_flip(stream, iterations=300_000, every=100):
    """The paper's whole performance run, read literally (Sec. 4): 300 x 300 lattice, J = 1,
    B = 0, 1500 replicas at T_i = 1 + 3i/|R|, 300,000 single-spin-flip iterations per
    replica, a swap iteration every 100 iterations. Timed from launch to completion."""
    import torch
    from paper_2512_03825_b300 import api
    from paper_2512_03825_b300 import workloads as W
    p = W.paper_problem()
    h = api.PTProblem(p.L, p.betas, seed=p.seed, stream=stream)
    h.flip(100, every)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    h.flip(iterations, every)
    b.record(stream)
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1e3
    h.close()
    flips = float(p.R) * iterations
    return {"value": flips / s, "unit": "single-spin-flip attempts/s", "seconds": s,
            "replicas": p.R, "iterations": iterations, "swap_every": every,
            "note": "the paper reports this run under 1 s on an A100 (CUDA version)"}


def bench_e2e(probs, sweeps, stream, world, steps=1):
    """The same step through the C ABI from host buffers: create every problem from host
    betas (tables copied to the device), run the batch, read energies, magnetisations,
    temperature maps and swap counters of every problem back in one transfer
    (pt_read_batch), destroy. One untimed step, then `steps` timed ones."""
    import torch
    from paper_2512_03825_b300 import api

    def step():
        hs = [api.PTProblem(p.L, p.betas, seed=p.seed, stream=stream) for p in probs]
        h2d = sum(h.device_bytes - h.L * h.L * ((h.R + 31) // 32) * 4 for h in hs)
        api.sweep_batch(hs, sweeps, 1)
        d2h = 0
        for r in api.read_batch(hs):
            d2h += sum(a.nbytes for a in r.values())
        for h in hs:
            h.close()
        return h2d, d2h

    step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        h2d, d2h = step()
    torch.cuda.synchronize()
    barrier(world)
    dt = max_over_ranks(time.perf_counter() - t0, world) / steps
    return {"value": _attempts(probs, sweeps) * world / dt, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "s_per_step": dt, "steps": steps}


def _oracle_rate(probs, sweeps_of, every_of, threads):
    """Attempts per second of the oracle, as it stands, on `threads` host threads over the
    given problems (each from creation for sweeps_of(p) sweeps)."""
    import oracle
    oracle.set_threads(threads)
    att = 0.0
    t0 = time.perf_counter()
    for p in probs:
        o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
        o.sweep(sweeps_of(p), every_of(p))
        att += float(p.L * p.L * p.R) * sweeps_of(p)
    dt = time.perf_counter() - t0
    return att / dt, dt, att


def cpu_baseline_plan(probs):
    """The oracle, as it stands, on the machine's host cores: the headline figure on a bounded
    sample of the batched workload (every 8th of the 256 problems, 100 sweeps each), and
    beside it the single-problem workloads (L = 16 and L = 128 in full, L = 1024 on its first
    10 sweeps), one core on a sample of L = 128, and the served stream on a 5% sample
    (every 20th request, at most 10 sweeps each; the whole stream's time extrapolated from
    its attempts)."""
    from paper_2512_03825_b300 import workloads as W
    threads = os.cpu_count() or 1
    sample = probs[:: max(1, len(probs) // 32)][:32]
    v, dt, _ = _oracle_rate(sample, lambda p: 100, lambda p: 1, threads)
    out = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "%d of the batched problems (every %d-th), 100 sweeps each, exchange "
                     "every sweep, %.1f s" % (len(sample), max(1, len(probs) // 32), dt)}
    plan = {}
    for name, sweeps in (("L16_R8", None), ("L128_R32", None), ("L1024_R64", 10)):
        p = W.SINGLE[name]
        sw = (lambda q: q.sweeps) if sweeps is None else (lambda q, k=sweeps: k)
        v1, dt1, _ = _oracle_rate([p], sw, lambda q: q.every, threads)
        plan[name] = {"value": v1, "sweeps": sw(p), "seconds": dt1,
                      "full_run": sweeps is None}
    p = W.SINGLE["L128_R32"]
    v1, dt1, _ = _oracle_rate([p], lambda q: 100, lambda q: q.every, 1)
    plan["L128_R32_one_core"] = {"value": v1, "sweeps": 100, "seconds": dt1, "cores": 1}
    reqs = W.serving_requests(n=2000, rate_per_s=1.0)
    samp = [r.problem for r in reqs[::20]]
    v1, dt1, att = _oracle_rate(samp, lambda q: min(10, q.sweeps), lambda q: q.every, threads)
    total = float(sum(r.problem.attempts for r in reqs))
    plan["serve_2000"] = {"value": v1, "requests": len(samp), "sweeps_each": "min(10, asked)",
                          "seconds": dt1, "extrapolated_total_s": total / v1}
    out["plan"] = plan
    return out


def run_single(args, rank, world, stream, sms):
    import torch
    from paper_2512_03825_b300 import api, autotune
    from paper_2512_03825_b300 import workloads as W
    p = W.SINGLE[args.single]
    h = api.PTProblem(p.L, p.betas, seed=p.seed, stream=stream)
    if args.sweep_strategy == "auto":
        if autotune.apply_single(h, p.L, p.R, p.J, p.h) is None:
            h.set_sweep_tuning(0)
    else:
        h.set_sweep_tuning({"launches": 1, "persistent": 2, "bands": 3}[args.sweep_strategy])
    shape = h.sweep_tuning()
    for _ in range(args.warmup):
        h.sweep(p.sweeps // 10, p.every)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        h.sweep(p.sweeps, p.every)
    b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    s = max_over_ranks(a.elapsed_time(b) / 1e3, world)
    per_step = float(p.L * p.L * p.R * p.sweeps)
    if h.sweep_tuning()[2] > 0:  # persistent: one cooperative launch per call
        launches = args.steps
    else:  # two half sweeps per sweep, an energy count and an exchange per swap iteration
        launches = args.steps * (2 * p.sweeps + 2 * (p.sweeps // p.every if p.every else 0))
    return {"metric": METRIC, "value": per_step * args.steps * world / s, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "single L=%d R=%d betas %.2f-%.2f, %d sweeps, exchange "
                                   "every %d, plain path" % (p.L, p.R, min(p.betas),
                                                             max(p.betas), p.sweeps, p.every),
                       "sweep_strategy": args.sweep_strategy,
                       "shape": {"strategy": shape[0], "words_per_thread": shape[1],
                                 "persistent_grid": shape[2]}},
            "clocks": clk, "gpu_launches": launches}


def run_flip(args, rank, world, stream):
    """The paper's performance run read as single-spin flips (Sec. 4.2): 300 x 300, J = 1,
    B = 0, 1500 replicas at T_i = 1 + 3i/|R|, args.iterations iterations per replica per
    step, a swap iteration every 100 iterations."""
    import torch
    from paper_2512_03825_b300 import api
    from paper_2512_03825_b300 import workloads as W
    p = W.paper_problem()
    h = api.PTProblem(p.L, p.betas, seed=p.seed, stream=stream)
    for _ in range(args.warmup):
        h.flip(min(args.iterations, 3000), 100)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        h.flip(args.iterations, 100)
    b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    s = max_over_ranks(a.elapsed_time(b) / 1e3, world)
    per_step = float(p.R) * args.iterations
    return {"metric": "single-spin-flip attempts/sec (all replicas, 1 B300)",
            "value": per_step * args.steps * world / s, "unit": "attempts/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "the paper's run as single flips: L=300, 1500 replicas, "
                                   "T_i = 1 + 3i/1500, %d iterations, swap every 100"
                                   % args.iterations},
            "clocks": clk, "gpu_launches": args.steps}


def run_converge(args, rank, world, stream):
    """Sweeps to convergence against L (Sec. 4.1, Fig. 3b), by the two-start reading of
    converge.py: the paper's ladder T_i = 1 + 3i/32 (32 temperatures), J = 1, B = 0, a swap
    iteration after every sweep, `--seeds` seeds per size; every hot/cold pair of runs
    advances in one batch until all its temperatures have converged (or its cap)."""
    import torch
    from paper_2512_03825_b300 import api
    from paper_2512_03825_b300 import converge as CV
    Ls = [int(x) for x in args.sizes.split(",")]
    seeds = [0x5EED4000 + rank * RANK_SEED_STRIDE + j for j in range(args.seeds)]
    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    clocks.start()
    t0 = time.perf_counter()
    details = {}
    res = CV.measure(api, Ls, seeds, R=32, every=1, stream=stream, details=details)
    torch.cuda.synchronize()
    wall = max_over_ranks(time.perf_counter() - t0, world)
    clk = clocks.stop()
    summ = CV.summarise(res, CV.default_caps(Ls))
    summ["slowest_temperature_index"] = CV.slowest_temperatures(details)
    return {"metric": "sweeps to converge against L (Fig. 3b): fitted exponent of the median",
            "value": summ.get("exponent_sweeps"), "unit": "exponent (t* ~ L^value sweeps)",
            "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * wall,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (random and ordered starts from the seed)",
            "config": {"workload": "convergence: L in %s, the paper's ladder with 32 "
                                   "temperatures, J=1, B=0, swap every sweep, %d seeds"
                                   % (args.sizes, args.seeds),
                       "criterion": "per temperature: first sweep with E(random start) <= "
                                    "E(ordered start), same seed; t* = last temperature"},
            "convergence": summ, "clocks": clk}


# ---------------------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    from paper_2512_03825_b300 import workloads as W
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    probs = rank_problems(0, args.problems, args.sweeps, 1, args.field)
    sample = probs[::16][:16]
    sweeps = 20
    for _ in range(max(0, min(args.warmup, 1))):
        o = oracle.OracleProblem(sample[0].L, sample[0].betas, seed=sample[0].seed)
        o.sweep(2, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for p in sample:
            o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
            o.sweep(sweeps, 1)
        times.append(time.perf_counter() - t0)
    att = _attempts(sample, sweeps)
    v = att * len(times) / sum(times)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic (same seeded problem mix)",
            "config": batched_config(args, _attempts(probs, args.sweeps)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "each step: 16 of the %d batched problems (every 16th), "
                                       "%d sweeps each, exchange every sweep"
                                       % (len(probs), sweeps)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

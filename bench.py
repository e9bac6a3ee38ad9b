#!/usr/bin/env python
"""Benchmark of the GB300 multi-objective Digital Annealer (MDA).

One *step* is one complete anneal of the workload: every replica runs all
I_max iterations of Alg. 3 (Sec. 3.3 of arXiv 2205.13399) -- parallel-trial
acceptance over all n^2 bits, one flip, archive update or archive jump --
through the C ABI.  Default workload: n = 25 (625-bit QUBO), 128 replicas,
I_max = 10^5, seed 0; synthetic instance (rounded Euclidean distances on a
100 x 100 grid, uniform [0, 99] flows with Gaussian-copula correlation 0.5).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload P25]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Prints one JSON line (rank 0).  ``value`` is replica-steps/s of the whole
job from CUDA-event kernel times (inputs resident); ``e2e`` is the same
metric through the public API with host matrices (instance upload, anneal,
merged non-dominated archive read-back) timed by wall clock.  Under torchrun
every rank anneals its own replica indices (weak scaling, no collective on
the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Algorithmic integer work of one bit-trial (one bit tested at one
# iteration): field update 2, Delta E of both objectives with the penalty
# term 10, acceptance penalty and threshold tests 6, ballot bookkeeping 2.
OPS_PER_BIT_TRIAL = 20
# INT32 lanes per SM (4 sub-partitions x 32 lanes issue one warp
# instruction per clock each).
INT_LANES_PER_SM = 128
L2_FLUSH_BYTES = 512 << 20

# DRAM bytes (read + write) of one annealing launch of the default workload,
# from one ncu capture per kernel, valid only for the kernel sources it was
# taken on (their SHA-256 below).
KERNEL_FILES = {
    "anneal_kernel": ("moda_kernel_body.cuh", "moda_kernel.cu", "moda_kernel_special.cu",
                      "moda_internal.h"),
    "warp_anneal_kernel": ("moda_warp.cu", "moda_device.cuh", "moda_internal.h"),
}
KERNEL_TRAFFIC = {
    "anneal_kernel": {"workload": "P25", "bytes": None, "sha256": None},
    "warp_anneal_kernel": {"workload": "P25", "bytes": 1052635392 + 1924999424,
                           "sha256": "53a5ceb321a40b0fe68edded14958ce48972a2441468e5ad548d69a129d1f59b"},
}


def kernel_sources_sha256(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_FILES[kernel]:
        with open(os.path.join(ROOT, "paper_2205_13399_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_traffic(kernel: str, workload: str, I_max: int, default_I_max: int):
    """DRAM bytes per launch when the stored capture matches this kernel,
    its sources and the workload, else None."""
    rec = KERNEL_TRAFFIC.get(kernel)
    if (rec is None or rec["bytes"] is None or workload != rec["workload"]
            or I_max != default_I_max or kernel_sources_sha256(kernel) != rec["sha256"]):
        return None
    return rec["bytes"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["moda", "reference"], default="moda")
    ap.add_argument("--workload", default="P25",
                    choices=["P8", "P25", "P50", "P75", "BATCH", "SERVE", "SBDA", "HVTRACE",
                             "QUBO"])
    ap.add_argument("--instances", type=int, default=512, help="BATCH: instances")
    ap.add_argument("--seq-instances", type=int, default=24,
                    help="BATCH / SERVE: requests also run one at a time for comparison")
    ap.add_argument("--requests", type=int, default=256, help="SERVE: requests")
    ap.add_argument("--rate", type=float, default=200.0, help="SERVE: arrivals per second")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fast-forward", action="store_true",
                    help="skip the extra fast-forward measurement of the single-instance line")
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--prefetch", type=int, default=0,
                    help="field-cache prefetch distance + 1 (0: automatic)")
    ap.add_argument("--field-cache", default="auto", choices=["auto", "on", "off"])
    ap.add_argument("--no-batch", action="store_true",
                    help="default run: skip the BATCH sub-measurement")
    ap.add_argument("--no-serve", action="store_true",
                    help="default run: skip the SERVE sub-measurement")
    ap.add_argument("--batch-seq-instances", type=int, default=512,
                    help="default run: BATCH instances also run one after another")
    ap.add_argument("--engine", default="auto", choices=["auto", "block", "warp"],
                    help="one thread block or one warp per replica (auto: warp when possible)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick block shape and prefetch distance by timed trials first")
    ap.add_argument("--no-autotune", action="store_true",
                    help="BATCH: keep the default block shapes (tuned per instance size otherwise)")
    ap.add_argument("--normalize", action="store_true",
                    help="QUBO normalisation (Sec. 4.2) in the acceptance test")
    ap.add_argument("--I-max", dest="I_max", type=int, default=None,
                    help="override the workload's iteration budget (profiling only)")
    return ap.parse_args(argv)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard(total_replicas: int, rank: int, world: int):
    """Weak scaling: every rank anneals ``total_replicas`` runs with its own
    replica indices [rank * total, (rank + 1) * total)."""
    return rank * total_replicas, total_replicas


def reduce_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(workload: str, budget_threads: int | None = None, first: int = 0):
    """The CPU oracle, as it stands, on the host cores: one replica per core
    (replica indices first, first + 1, ... modulo the workload's replica
    count), each for the workload's full I_max (the whole cooling
    schedule)."""
    import oracle
    from paper_2205_13399_gb300 import inputs
    inst = inputs.workload_instance(workload)
    run = inputs.WORKLOAD_RUN[workload]
    cores = budget_threads or (os.cpu_count() or 1)
    reps = min(cores, run["replicas"])
    rows = [(first + k) % run["replicas"] for k in range(reps)]
    I_max = run["I_max"]
    oi = oracle.Instance(inst.F1, inst.F2, inst.D)
    t0 = time.perf_counter()
    oracle.run(oi, I_max=I_max, replicas=rows, seed=run["seed"], threads=cores)
    dt = time.perf_counter() - t0
    value = reps * I_max / dt
    return {"value": value, "unit": "replica-steps/s", "cores": min(cores, reps),
            "kind": "oracle",
            "sample": f"{reps} of {run['replicas']} replicas (from index {rows[0]}), "
                      f"full I_max={I_max}, {dt:.1f} s wall"}, dt


def int_peak(sm_max_mhz, sms):
    """Measured INT32 lane-op peak (moda_probe_int_peak) with the derived one."""
    from paper_2205_13399_gb300 import moda
    measured, _ = moda.probe_int_peak(20000)
    smem, _ = moda.probe_smem_peak(20000)
    derived = sms * INT_LANES_PER_SM * sm_max_mhz * 1e6
    return measured, derived, smem


def roofline_line(ops, seconds, sms, sm_max_mhz, per_unit):
    measured, derived, smem = int_peak(sm_max_mhz, sms)
    achieved = ops / seconds
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": measured / 1e12,
            "unit": "Tops/s", "frac": achieved / measured, "traffic": None,
            "kernel": "anneal_kernel", "per_unit": per_unit,
            "peak_source": "measured: moda_probe_int_peak (INT32 lane-ops/s, all SMs)",
            "peak_derived": derived / 1e12,
            "smem_peak_GBps": smem / 1e9}


def workload_config(workload, inst, run, extra=None):
    cfg = {"workload": f"{workload}: bi-objective QAP n={inst.n} ({inst.n * inst.n}-bit QUBO), "
                       f"{run['replicas']} replicas, I_max={run['I_max']}",
           "n": inst.n, "bits": inst.n * inst.n, "replicas": run["replicas"],
           "I_max": run["I_max"], "seed": run["seed"], "accept": "strict",
           "archive": "explore", "escape": "archive",
           "schedule": {"delta0": 1e9, "deltaf": 1e4, "xi": 1e-3},
           "l2": "flushed between timed steps (512 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2205_13399_gb300 import inputs
    inst = inputs.workload_instance(args.workload)
    run = inputs.WORKLOAD_RUN[args.workload]
    work, secs = 0, 0.0
    base = None
    cores = os.cpu_count() or 1
    reps = min(cores, run["replicas"])
    for k in range(args.warmup + args.steps):
        # step k runs the next block of replica indices, so consecutive
        # steps cover every replica of the workload
        base, dt = cpu_baseline(args.workload, first=(k * reps) % run["replicas"])
        if k >= args.warmup:
            work += reps * run["I_max"]
            secs += dt
    value = work / secs
    line = {
        "impl": "reference", "metric": "replica-steps/s", "value": value,
        "unit": "replica-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": workload_config(args.workload, inst, run,
                                  {"parallelism": f"replicas x{args.gpus} GPU(s)"}),
        "cpu_baseline": {**base, "value": value,
                         "sample": f"each step: {reps} of {run['replicas']} replicas at the "
                                   f"full I_max={run['I_max']}, consecutive steps taking the "
                                   "next replica indices"},
        "e2e": {"value": value, "unit": "replica-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "note": "the CPU oracle on the host cores; each step is a bounded sample of the "
                "workload (see cpu_baseline.sample) and ms_per_step is its measured wall time",
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_measure(args, steps: int, warmup: int, seq_instances: int):
    """BATCH: 512 instances of uneven size (n uniform in [10, 75]), 32
    replicas each, I_max = 10^5, all enqueued by one moda_anneal_batch call
    (one CUDA graph launch) per step; the first ``seq_instances`` instances
    also run as plain launches one after another for comparison.  Returns
    the measurement as a dict."""
    import torch
    from paper_2205_13399_gb300 import inputs, moda
    dev = torch.device("cuda", torch.cuda.current_device())
    I_max = args.I_max if args.I_max is not None else 100_000
    qis = inputs.batch_instances(args.instances)
    insts = [moda.Instance(q.F1, q.F2, q.D) for q in qis]
    params = [moda.make_params(replicas=32, I_max=I_max, seed=k, engine=args.engine)
              for k in range(len(qis))]
    warm = [moda.make_params(replicas=32, I_max=min(I_max, 1000), seed=k, engine=args.engine)
            for k in range(len(qis))]
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if args.autotune:  # untimed: one tuning per instance size, shared by its instances
        t0 = time.perf_counter()
        by_n = {}
        for q, inst, p, pw in zip(qis, insts, params, warm):
            if q.n not in by_n:
                best, _ = moda.autotune(inst, params=p, trial_iters=1000, stream=stream)
                by_n[q.n] = (best.block_threads, best.prefetch)
            for pp in (p, pw):
                pp.block_threads, pp.prefetch = by_n[q.n]
        tuned = {"sizes": len(by_n), "tuning_s": time.perf_counter() - t0,
                 "trial_iters": 1000,
                 "shapes": {str(n): list(v) for n, v in sorted(by_n.items())}}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def batch(ps, subset=None):
        ii = insts if subset is None else insts[:subset]
        pp = ps if subset is None else ps[:subset]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        runs = moda.anneal_batch(ii, pp, stream=stream)
        b.record(stream)
        b.synchronize()
        for r in runs:
            r.wait()
            r.close()
        return a.elapsed_time(b)

    for _ in range(warmup):
        batch(warm)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        ms.append(batch(params))
    clk = clocks.stop()
    rep_steps = sum(p.replicas for p in params) * I_max
    value = rep_steps * steps / (sum(ms) / 1e3)
    k = min(seq_instances, len(insts))
    seq_ms = 0.0
    for i in range(k):
        r = moda.anneal(insts[i], params[i], stream=stream).wait()
        seq_ms += r.elapsed_ms()
        r.close()
    sub_ms = statistics.mean(ms) if k in (0, len(insts)) else batch(params, subset=k)
    # end to end: instance upload, the batch, merged fronts read back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ii = [moda.Instance(q.F1, q.F2, q.D) for q in qis]
    runs = moda.anneal_batch(ii, params, stream=stream)
    npts = 0
    for r in runs:
        npts += len(r.wait().read_archive(-1, perms=False))
        r.close()
    e2e_s = time.perf_counter() - t0
    h2d = sum(3 * q.n * q.n * 4 for q in qis)
    d2h = npts * 40
    props = torch.cuda.get_device_properties(dev)
    ops = sum(p.replicas * I_max * q.n * q.n for p, q in zip(params, qis)) * OPS_PER_BIT_TRIAL
    roofline = roofline_line(ops, statistics.mean(ms) / 1e3, props.multi_processor_count,
                             clk.get("sm_max_mhz") or 2070.0,
                             f"{OPS_PER_BIT_TRIAL} int32 lane-ops per bit-trial")
    roofline["kernel"] = "warp_anneal_kernel" if args.engine != "block" else "anneal_kernel"
    ns = [q.n for q in qis]
    return {
        "metric": "replica-steps/s", "value": value, "unit": "replica-steps/s", "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": f"BATCH: {len(qis)} bi-objective QAP instances, n uniform in "
                               f"[{min(ns)}, {max(ns)}], 32 replicas each, I_max={I_max}, "
                               "one moda_anneal_batch call (one CUDA graph launch) per step",
                   "instances": len(qis), "replicas_each": 32, "I_max": I_max,
                   "engine": args.engine,
                   "mean_bits": statistics.mean(n * n for n in ns),
                   "warmup_I_max": min(I_max, 1000),
                   "l2": "flushed between timed steps (512 MiB write)",
                   **({"autotuned": tuned} if tuned else {})},
        "bit_trials_per_s": value * statistics.mean(n * n for n in ns),
        "vs_sequential": None if k == 0 else {
            "instances": k, "batched_ms": sub_ms, "sequential_ms": seq_ms,
            "speedup": seq_ms / sub_ms,
            "what": "the same instances as plain moda_anneal launches one after another "
                    "(sum of their kernel times) against the batch"},
        "e2e": {"value": rep_steps / e2e_s, "unit": "replica-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": 1},
        "gpu_launches": None, "roofline": roofline, "clocks": clk,
    }


def run_batch(args):
    line = batch_measure(args, args.steps, args.warmup, args.seq_instances)
    print(json.dumps(line), flush=True)
    return 0


def serve_measure(args, rate: float, requests: int, warmup: int, seq_instances: int,
                  batch_same: bool = False):
    """SERVE: Poisson arrivals (``rate`` per second) of solves with n in
    {20, 30, 50, 75} and I_max in {10^4, 10^5}, 32 replicas each, through
    the serving queue; latency is arrival to the poll that returns the
    finished run.  Returns the measurement as a dict."""
    import numpy as np
    import torch
    from paper_2205_13399_gb300 import inputs, moda
    reqs = inputs.serving_requests(requests, rate_per_s=rate)
    warm = inputs.serving_requests(max(warmup, 1) * 4, rate_per_s=rate, index0=10_000_000)

    def serve(rs):
        srv = moda.Server()
        t0 = time.perf_counter()
        pending, lat, done_t = {}, [], []
        kernel_ms = []
        most = 0
        nxt = 0
        while nxt < len(rs) or pending:
            now = time.perf_counter() - t0
            while nxt < len(rs) and rs[nxt].arrival_s <= now:
                q = rs[nxt]
                inst = moda.Instance(q.instance.F1, q.instance.F2, q.instance.D)
                t = srv.submit(inst, replicas=32, I_max=q.I_max, seed=q.seed,
                               engine=args.engine)
                pending[t] = (q, inst)
                nxt += 1
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    q, inst = pending.pop(t)
                    r.read_archive(-1, perms=False)
                    kernel_ms.append(r.elapsed_ms())
                    fin = time.perf_counter() - t0
                    lat.append(fin - q.arrival_s)
                    done_t.append(fin)
                    r.close()
            most = max(most, srv.info()["running"])
            time.sleep(0.0005)
        srv.close()
        return np.array(lat), max(done_t), kernel_ms, most

    for _ in range(warmup):
        serve(warm[:4])
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    lat, span, _, most = serve(reqs)
    clk = clocks.stop()
    value = len(reqs) / span
    # the first k requests both ways: served (as they arrive) and one at a
    # time, each solve waited for before the next starts
    k = min(seq_instances, len(reqs))
    vs = None
    if k > 0:
        _, span_k, served_ms, _ = serve(reqs[:k])
        t0 = time.perf_counter()
        alone_ms = []
        for q in reqs[:k]:
            inst = moda.Instance(q.instance.F1, q.instance.F2, q.instance.D)
            r = moda.anneal(inst, replicas=32, I_max=q.I_max, seed=q.seed,
                            engine=args.engine).wait()
            r.read_archive(-1, perms=False)
            alone_ms.append(r.elapsed_ms())
            r.close()
        seq_span = time.perf_counter() - t0
        vs = {"requests": k, "served_s": span_k, "one_at_a_time_s": seq_span,
              "speedup": seq_span / span_k,
              "kernel_ms_served_over_alone": sum(served_ms) / max(sum(alone_ms), 1e-9)}
    work = sum(32 * q.I_max for q in reqs)
    # the same requests as one batch launch (all known in advance): the
    # throughput the GPU gives this mix of sizes and schedules
    same = None
    if batch_same:
        insts = [moda.Instance(q.instance.F1, q.instance.F2, q.instance.D) for q in reqs]
        prms = [moda.make_params(replicas=32, I_max=q.I_max, seed=q.seed, engine=args.engine)
                for q in reqs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        runs = moda.anneal_batch(insts, prms)
        for r in runs:
            r.wait()
        bspan = time.perf_counter() - t0
        for r in runs:
            r.close()
        same = {"batch_s": bspan, "batch_replica_steps_per_s": work / bspan,
                "served_over_batch_time": span / bspan}
    return {
        "metric": "bQAP solves/s", "value": value, "unit": "solves/s", "n_gpus": 1,
        "steps": 1, "warmup": warmup, "ms_per_step": span * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": f"SERVE: {len(reqs)} requests, Poisson {rate:g}/s, n in "
                               "{20, 30, 50, 75}, I_max in {1e4, 1e5}, 32 replicas each",
                   "requests": len(reqs), "rate_per_s": rate, "engine": args.engine,
                   "admission": "HBM budget = free memory less max(1/8, 1 GiB)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                       "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
        "most_running": most,
        "replica_steps_per_s": work / span,
        "vs_one_at_a_time": vs,
        "vs_same_requests_batched": same,
        "e2e": {"value": value, "unit": "solves/s",
                "h2d_bytes_per_step": sum(3 * q.instance.n ** 2 * 4 for q in reqs),
                "d2h_bytes_per_step": None, "note": "serving is end to end by construction"},
        "gpu_launches": len(reqs), "clocks": clk,
    }


def serve_both(args, requests: int, warmup: int, seq_instances: int):
    """The SERVE config's rate, then 70 % of the capacity it measured, so the
    latency of the second line is the server's own rather than queueing."""
    line = serve_measure(args, args.rate, requests, warmup, seq_instances, batch_same=True)
    cap = line["value"]
    if cap * 0.7 < args.rate:
        sus = serve_measure(args, 0.7 * cap, requests, 0, 0)
        line["at_70pct_capacity"] = {
            "rate_per_s": 0.7 * cap, "value": sus["value"], "unit": "solves/s",
            "latency_ms": sus["latency_ms"], "most_running": sus["most_running"],
            "clocks": sus["clocks"]}
    return line


def run_serve(args):
    line = serve_both(args, args.requests, args.warmup, args.seq_instances)
    print(json.dumps(line), flush=True)
    return 0


def hv_norm(points, lo, hi):
    """Normalised 2-D hypervolume (minimisation) of ``points`` in the box
    [lo, hi] scaled to [0, 1]^2, reference point (1.1, 1.1)."""
    pts = sorted(((p[0] - lo[0]) / max(hi[0] - lo[0], 1), (p[1] - lo[1]) / max(hi[1] - lo[1], 1))
                 for p in points)
    hv, prev2 = 0.0, 1.1
    for a, b in pts:
        if b < prev2:
            hv += (1.1 - a) * (prev2 - b)
            prev2 = b
    return hv


def run_sbda(args):
    """SB-DA (Alg. 2: eleven scalarised DA runs, one batch launch) against
    MDA (Alg. 3) on the P25 instance in the paper's setting (Sec. 4.2, 5.1:
    normalised QUBOs, I_max = 0.25 m^2, delta0 = 1e9, delta_f = 1e4,
    xi = 0.001, beta = delta0 / I_max), same replicas per run: the paper's
    comparison of the two (Table 3), with both fronts' normalised
    hypervolume over the union's cost range.  The same comparison on the
    integer QUBOs is reported beside it."""
    import torch
    from paper_2205_13399_gb300 import inputs, moda
    dev = torch.device("cuda", torch.cuda.current_device())
    qi = inputs.workload_instance("P25")
    run = dict(inputs.WORKLOAD_RUN["P25"])
    m = qi.n * qi.n
    I_max = args.I_max if args.I_max is not None else m * m // 4
    R = run["replicas"]
    sched = dict(delta0=1e9, deltaf=1e4, xi=1e-3)
    inst = moda.Instance(qi.F1, qi.F2, qi.D)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), out

    def compare(normalize, steps, warmup):
        def sbda():
            return moda.sbda(inst, replicas=R, I_max=I_max, seed=run["seed"],
                             normalize=normalize, stream=stream, **sched)

        def mda():
            r = moda.anneal(inst, replicas=R, I_max=I_max, seed=run["seed"],
                            normalize=normalize, stream=stream, **sched)
            r.wait()
            return r

        for _ in range(warmup):
            for x in sbda()[0]:
                x.close()
            mda().close()
        s_ms, m_ms = [], []
        for _ in range(steps):
            ms, (runs, front_s) = timed(sbda)
            s_ms.append(ms)
            ms, r = timed(mda)
            m_ms.append(ms)
            front_m = [(p["c1"], p["c2"]) for p in r.read_archive(-1) if p["feasible"]]
            r.close()
            for x in runs:
                x.close()
        fs = [(p["c1"], p["c2"]) for p in front_s]
        allp = fs + front_m
        lo = (min(p[0] for p in allp), min(p[1] for p in allp))
        hi = (max(p[0] for p in allp), max(p[1] for p in allp))
        sb, md = statistics.mean(s_ms), statistics.mean(m_ms)
        return {"normalised": normalize, "sbda_ms": sb, "mda_ms": md,
                "sbda_over_mda_time": sb / md, "mda_engine": "block" if normalize else "warp",
                "sbda_front_points": len(fs), "mda_front_points": len(front_m),
                "hv_sbda": hv_norm(fs, lo, hi), "hv_mda": hv_norm(front_m, lo, hi)}

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    main = compare(True, args.steps, args.warmup)
    integer = compare(False, 1, 1)
    clk = clocks.stop()
    sb = main["sbda_ms"]
    value = 11 * R * I_max / (sb / 1e3)
    line = {
        "metric": "replica-steps/s", "value": value, "unit": "replica-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sb,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
        "data": "synthetic",
        "config": {"workload": f"SBDA: SB-DA (11 weights, Alg. 2) vs MDA (Alg. 3) on P25, "
                               f"normalised QUBOs, {R} replicas, I_max={I_max} per run",
                   "weights": 11, "replicas": R, "I_max": I_max, **sched,
                   "beta": "delta0 / I_max",
                   "l2": "flushed before each timed solve (512 MiB write)"},
        "vs_mda": main,
        "integer_qubos": integer,
        "e2e": {"value": value, "unit": "replica-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": None, "note": "front read-back inside the timed call"},
        "gpu_launches": 12 * args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_hvtrace(args):
    """Fig. mdasl: the hypervolume of the merged archive after every K
    iterations, strict against lenient acceptance (explorative archive), on
    the P25 instance; feasible points' costs normalised to [1, 2] over both
    runs, reference point (2.1, 2.1), so 1.21 is the largest possible."""
    import torch
    from paper_2205_13399_gb300 import inputs, moda
    qi = inputs.workload_instance("P25")
    run = dict(inputs.WORKLOAD_RUN["P25"])
    if args.I_max is not None:
        run["I_max"] = args.I_max
    R, I_max = run["replicas"], run["I_max"]
    K = max(1, I_max // 100)
    inst = moda.Instance(qi.F1, qi.F2, qi.D)
    out, ms = {}, {}
    for _ in range(args.warmup):
        moda.anneal(inst, replicas=R, I_max=min(I_max, 2000), seed=run["seed"]).wait().close()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for acc in ("strict", "lenient"):
        r = moda.anneal(inst, replicas=R, I_max=I_max, seed=run["seed"], accept=acc,
                        snapshot_every=K).wait()
        ms[acc] = r.elapsed_ms()
        out[acc] = [[(p["c1"], p["c2"]) for p in r.read_archive(snapshot=j, perms=False)
                     if p["feasible"]] for j in range(I_max // K)]
        r.close()
    # the snapshot cost against the same engine without snapshots (the
    # block engine: snapshots are one of its options), and the warp engine
    # a run without snapshots takes by default
    plain = moda.anneal(inst, replicas=R, I_max=I_max, seed=run["seed"], engine="block").wait()
    plain_ms = plain.elapsed_ms()
    plain.close()
    plain = moda.anneal(inst, replicas=R, I_max=I_max, seed=run["seed"]).wait()
    warp_ms = plain.elapsed_ms()
    plain.close()
    clk = clocks.stop()
    allp = [p for acc in out for f in out[acc] for p in f]
    lo = (min(p[0] for p in allp), min(p[1] for p in allp)) if allp else (0, 0)
    hi = (max(p[0] for p in allp), max(p[1] for p in allp)) if allp else (1, 1)
    hv = {acc: [hv_norm(f, lo, hi) if f else 0.0 for f in out[acc]] for acc in out}

    def reach(curve, frac=0.95):
        top = curve[-1]
        for j, v in enumerate(curve):
            if v >= frac * top:
                return (j + 1) * K
        return None

    line = {
        "metric": "replica-steps/s", "value": R * I_max / (ms["strict"] / 1e3),
        "unit": "replica-steps/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": ms["strict"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"HVTRACE: P25, {R} replicas, I_max={I_max}, archive snapshot "
                               f"every {K} iterations, strict vs lenient (explore)",
                   "snapshot_every": K},
        "hv_final": {acc: hv[acc][-1] for acc in hv},
        "iterations_to_95pct_hv": {acc: reach(hv[acc]) for acc in hv},
        "hv_every_10_snapshots": {acc: [round(v, 4) for v in hv[acc][9::10]] for acc in hv},
        "snapshot_overhead": {"ms_with": ms["strict"], "ms_plain": plain_ms,
                              "engine": "block",
                              "ms_default_engine_without_snapshots": warp_ms},
        "gpu_launches": 2, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_qubo(args):
    """Explicit QUBOs with K = 3 objectives: dense random m = 1024 matrices,
    128 replicas, I_max = 10^5 (the stored-P generalisation of the path)."""
    import torch
    from paper_2205_13399_gb300 import inputs, moda
    dev = torch.device("cuda", torch.cuda.current_device())
    K, m, R = 3, 1024, 128
    I_max = args.I_max if args.I_max is not None else 100_000
    Q = inputs.random_qubo(K, m)
    q = moda.Qubo(Q)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    kw = dict(replicas=R, I_max=I_max, seed=0)
    for _ in range(args.warmup):
        q.anneal(stream=stream, **dict(kw, I_max=min(I_max, 2000))).wait().close()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        r = q.anneal(stream=stream, **kw).wait()
        ms.append(r.elapsed_ms())
        r.close()
    clk = clocks.stop()
    value = R * I_max * args.steps / (sum(ms) / 1e3)
    t0 = time.perf_counter()
    q2 = moda.Qubo(Q)
    r = q2.anneal(stream=stream, **kw).wait()
    res = r.read()
    e2e_s = time.perf_counter() - t0
    r.close()
    line = {
        "metric": "replica-steps/s", "value": value, "unit": "replica-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": f"QUBO: K={K} dense random QUBOs, m={m} bits, {R} replicas, "
                               f"I_max={I_max}", "K": K, "bits": m, "replicas": R,
                   "I_max": I_max, "l2": "flushed between timed steps (512 MiB write)"},
        "bit_trials_per_s": value * m,
        "e2e": {"value": R * I_max / e2e_s, "unit": "replica-steps/s",
                "h2d_bytes_per_step": int(Q.nbytes),
                "d2h_bytes_per_step": int(sum(v.nbytes for v in res.values())), "steps": 1},
        "gpu_launches": args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_env()
    import numpy as np
    import torch
    if args.workload in ("BATCH", "SERVE", "SBDA", "HVTRACE", "QUBO"):
        if world > 1:
            raise SystemExit("BATCH, SERVE, SBDA, HVTRACE and QUBO run on one GPU")
        torch.cuda.set_device(local)
        return {"BATCH": run_batch, "SERVE": run_serve, "SBDA": run_sbda,
                "HVTRACE": run_hvtrace, "QUBO": run_qubo}[args.workload](args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2205_13399_gb300 import inputs, moda

    inst_np = inputs.workload_instance(args.workload)
    run = dict(inputs.WORKLOAD_RUN[args.workload])
    if args.I_max is not None:
        run["I_max"] = args.I_max
    R, I_max = run["replicas"], run["I_max"]
    base, R = shard(R, rank, world)
    m = inst_np.n * inst_np.n
    g = moda.Instance(inst_np.F1, inst_np.F2, inst_np.D)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    kw = dict(replicas=R, replica_base=base, I_max=I_max, seed=run["seed"],
              block_threads=args.block_threads, prefetch=args.prefetch,
              field_cache=args.field_cache, normalize=args.normalize, engine=args.engine)
    tuned = None
    if args.autotune:  # untimed: trials on the cold end of the schedule
        best, trial_ms = moda.autotune(g, **kw)
        kw.update(block_threads=best.block_threads, prefetch=best.prefetch)
        tuned = {"block_threads": best.block_threads, "prefetch": best.prefetch,
                 "trial_ms": trial_ms}

    def step():
        r = moda.anneal(g, stream=stream, **kw).wait()
        ms = r.elapsed_ms()
        r.close()
        return ms, None

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    kernel_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ms, _ = step()
        kernel_ms.append(ms)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = reduce_max(sum(kernel_ms), world, dev)
    rep_steps_all = R * I_max * args.steps * world
    value = rep_steps_all / (total_ms / 1e3)

    # The exact shortcut (moda_params.fast_forward), timed the same way
    # but reported beside the full-work headline: the results are those of
    # the full run, while the iterations after every archive member is
    # known unable to accept are settled without being executed.
    ff_line = None
    if not args.no_fast_forward and not args.normalize:
        ff_ms, skipped = [], 0
        for k in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            r = moda.anneal(g, stream=stream, fast_forward=True,
                            **{**kw, "engine": "block"}).wait()
            if k >= args.warmup:
                ff_ms.append(r.elapsed_ms())
                skipped += int(r.read().stats[:, 6].sum())
            r.close()
        ff_total = reduce_max(sum(ff_ms), world, dev)
        ff_line = {"value": rep_steps_all / (ff_total / 1e3), "unit": "replica-steps/s",
                   "ms_per_step": ff_total / args.steps,
                   "executed_frac": 1.0 - skipped / float(R * I_max * args.steps),
                   "what": "moda_params.fast_forward = 1: identical results (parity-tested "
                           "against the oracle's full run); not the headline"}

    # End to end through the public API with host buffers.
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(1, min(args.steps, 3))
    h2d = 3 * m * 4  # Fs1, Fs2, D uploaded as int32 by moda_create_instance
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    npts = 0
    for _ in range(e2e_steps):
        gi = moda.Instance(inst_np.F1, inst_np.F2, inst_np.D)
        r = moda.anneal(gi, stream=stream, **kw).wait()
        front = r.read_archive(-1)
        npts = len(front)
        r.close()
        gi.close()
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
    W = (m + 31) // 32
    s = m
    d2h = R * 4 + R * s * 16 + npts * W * 4
    e2e_value = R * I_max * e2e_steps * world / e2e_s

    # Roofline of the annealing kernel: integer issue bound.
    props = torch.cuda.get_device_properties(dev)
    sm_max_mhz = clk.get("sm_max_mhz") or 2070.0
    ops_per_launch = R * I_max * m * OPS_PER_BIT_TRIAL
    roofline = roofline_line(ops_per_launch, statistics.mean(kernel_ms) / 1e3,
                             props.multi_processor_count, sm_max_mhz,
                             f"{OPS_PER_BIT_TRIAL} int32 lane-ops per bit-trial")
    roofline["kernel"] = "anneal_kernel" if args.engine == "block" else "warp_anneal_kernel"
    roofline["traffic"] = kernel_traffic(
        roofline["kernel"], args.workload, I_max, inputs.WORKLOAD_RUN[args.workload]["I_max"])
    if roofline["traffic"] is not None:
        roofline["traffic_unit"] = "bytes per launch (ncu dram__bytes_read + write)"

    line = {
        "metric": "replica-steps/s", "value": value, "unit": "replica-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(args.workload, inst_np, run,
                                  {"parallelism": f"replicas x{world} GPU(s)",
                                   **({"autotuned": tuned} if tuned else {})}),
        "bit_trials_per_s": value * m,
        "e2e": {"value": e2e_value, "unit": "replica-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": args.steps,
        "roofline": roofline,
        "clocks": clk,
    }
    if ff_line is not None:
        line["fast_forward"] = ff_line
    if rank == 0 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(args.workload)
        line["cpu_baseline"] = cb
    # The metric's other two configs, measured in the same default run: the
    # batched launch of 512 instances of uneven n and the serving queue.
    if rank == 0:
        print(json.dumps({k: line[k] for k in ("value", "ms_per_step", "e2e")}),
              file=sys.stderr, flush=True)
    if world == 1 and args.workload == "P25" and not args.no_batch:
        line["batch"] = batch_measure(args, 1, 1, args.batch_seq_instances)
        print(json.dumps({"batch": line["batch"]}), file=sys.stderr, flush=True)
    if world == 1 and args.workload == "P25" and not args.no_serve:
        line["serve"] = serve_both(args, args.requests, 1, args.seq_instances)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

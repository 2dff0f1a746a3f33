"""Benchmark of the GB300-native MDFS information-gain scan.

One step = one MDFS scan job on the synthetic parity-structured data with
Madelon's shapes (N = 2000 objects, M = 500 variables, binary decision):
the k = 2 scan and the k = 3 scan, each over 30 random discretisations into
2 classes (range 0.5, pseudocount xi 0.25).  The metric is unordered
tuple x discretisation evaluations per second:
    (C(500, 2) + C(500, 3)) * 30 = 6.249e8 evaluations per step.

Default arm: inputs resident in HBM, each step timed with CUDA events on the
launching stream, L2 flushed (512 MB write) between steps.  ``e2e`` repeats
the steps through the C ABI with pinned host inputs and host outputs.  The
same JSON line also carries the measured tensor-core and shared-memory rates
of the GPU (``peaks``), the roofline of the k = 3 kernel against the measured
E4M3 rate, and the other configurations (``configs``: the 200 x 50 XOR case,
k = 1 and k = 2 on the parity data, the batched 64-job workload), each timed
and compared with the FP64 oracle on sampled variables.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (the method has no other reference implementation here).

Multi-GPU (torchrun): one job's tuple tiles are split over the ranks
(mdfs_max_ig_shard) and the packed max keys merged by one NCCL all-reduce
(MAX) of 8 M bytes: strong scaling, value = the job's evaluations / max rank
time.  ``--independent`` runs an independent job per rank instead (weak
scaling, no collective).  ``--shard`` takes the sharded path on one GPU too.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_OBJ, M_VAR, DISC, DIV, RANGE, XI = 2000, 500, 30, 1, 0.5, 0.25
METRIC = "k-tuple*discretization IG evals/sec (k=2,3; N=2000, M=500)"
UNIT = "tuple*disc/s"
WORKLOAD = "mdfs_scan_parity_N2000_M500_k2+k3_D30_c2"


def _units():
    return math.comb(M_VAR, 2) * DISC + math.comb(M_VAR, 3) * DISC


def _bf16_burst_peak():
    """Measured dense bf16 burst peak (TF/s) of this machine's GPUs, with its provenance."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def _use_small_case(n_disc: int = 2):
    """A reduced case of the same kernels for profiler captures (M = 500, n_disc discretisations)."""
    global M_VAR, DISC, WORKLOAD
    M_VAR, DISC = 500, n_disc
    WORKLOAD = f"mdfs_scan_parity_N2000_M500_k2+k3_D{n_disc}_c2 (profiling case)"


def _config(extra=None):
    cfg = {"workload": WORKLOAD, "N": N_OBJ, "M": M_VAR, "k": [2, 3], "discretizations": DISC,
           "divisions": DIV, "range": RANGE, "pc_xi": XI, "l2": "flushed (512 MB write) between timed steps",
           "data": "synthetic Madelon-shaped 5-bit parity set (seeded numpy PCG64)"}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to MDFS_BENCH_LOG_DIR when set, else to the system temp directory
        log_dir = os.environ.get("MDFS_BENCH_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class BusySampler:
    """nvidia-smi utilization.gpu (the share of each sample period in which a
    kernel ran) every 100 ms over a region: mean and median percent."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        log_dir = os.environ.get("MDFS_BENCH_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"busy_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", "--query-gpu=utilization.gpu",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        vals = []
        for line in open(self.path):
            try:
                vals.append(float(line.strip()))
            except ValueError:
                continue
        if not vals:
            return None
        return {"mean_pct": float(np.mean(vals)), "median_pct": float(np.median(vals)), "samples": len(vals)}


# ----------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(n2: int, n3: int, seed: int = 11, n_disc: int = None):
    """Times the FP64 oracle on n2 variables at k=2 and n3 variables at k=3
    (full partner scans over the first n_disc of the 30 discretisations,
    default all).  Returns (unordered tuple*disc equivalents processed,
    seconds, threads)."""
    import oracle
    from paper_1811_00631_gb300 import synth
    ds = synth.madelon_like()
    nd = DISC if n_disc is None else max(1, min(DISC, n_disc))
    t0 = time.perf_counter()
    codes = oracle.discretize(ds.x, DIV, nd, RANGE, seed)  # the first nd discretisations
    if n2:
        oracle.max_ig(codes, ds.y, DIV + 1, 2, XI, variables=np.arange(n2, dtype=np.int32))
    if n3:
        oracle.max_ig(codes, ds.y, DIV + 1, 3, XI, variables=np.arange(n3, dtype=np.int32))
    dt = time.perf_counter() - t0
    # each variable's scan covers C(M-1, k-1) * D (variable, partner set) roles;
    # an unordered k-tuple carries k roles
    units = n2 * (M_VAR - 1) * nd / 2 + n3 * math.comb(M_VAR - 1, 2) * nd / 3
    return units, dt, oracle.num_threads()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    n3 = max(1, threads)  # one k = 3 variable per host thread
    n2 = 64
    for _ in range(args.warmup):
        oracle_sample(n2, 0)
    # each step is a bounded sample: the discretisations per step are chosen
    # so that the timed steps take about two minutes in all (the rate,
    # tuple*disc/s, does not depend on how many discretisations a sample has)
    _, t1, _ = oracle_sample(n2, n3, n_disc=1)
    n_disc = int(max(1, min(DISC, (120.0 / max(args.steps, 1)) / max(t1, 1e-3))))
    times, units = [], 0.0
    for _ in range(args.steps):
        u, dt, _ = oracle_sample(n2, n3, n_disc=n_disc)
        times.append(dt)
        units += u
    total = sum(times)
    value = units / total
    sample = (f"{n2} variables at k=2 and {n3} at k=3, each a full partner scan over "
              f"{n_disc} of the {DISC} discretisations of the 2000x500 data, per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config({"oracle": "FP64 brute-force C (OpenMP)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1811_00631_gb300 import build, mdfs, synth

    from paper_1811_00631_gb300 import shard as shard_mod
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # sharded: every rank scans its share of one job's tuple tiles and the keys
    # are merged by one all-reduce (MAX) of 8 M bytes; independent: one job per rank
    sharded = args.shard or (world > 1 and not args.independent)
    ds = synth.madelon_like(M=max(M_VAR, 20), seed=2 if sharded else 2 + rank)
    x = torch.from_numpy(ds.x).to(dev)
    y = torch.from_numpy(ds.y).to(dev)
    M = M_VAR
    outs = {k: (torch.empty(M, dtype=torch.float32, device=dev), torch.empty((M, max(k - 1, 1)), dtype=torch.int32,
                                                                              device=dev),
                torch.empty(M, dtype=torch.int32, device=dev)) for k in (2, 3)}
    keys_t = {k: torch.empty(M, dtype=torch.int64, device=dev) for k in (2, 3)}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    launches = [0]

    def scan(xx, yy, k, seed, out):
        if sharded:
            mdfs.max_ig_shard(xx, yy, k, DIV, DISC, RANGE, XI, seed, shard=rank, n_shards=world, keys_out=keys_t[k])
            n = mdfs.last_launch_count()
            if world > 1:
                shard_mod.allreduce_max_device(keys_t[k])
            res = mdfs.decode_keys(keys_t[k], k, out=out if out is not None and hasattr(out[0], "is_cuda") else None)
            launches[0] += n + mdfs.last_launch_count()
            return res
        res = mdfs.max_ig(xx, yy, k, DIV, DISC, RANGE, XI, seed, out=out)
        launches[0] += mdfs.last_launch_count()
        return res

    def step(seed):
        if sharded:
            for k in (2, 3):
                scan(x, y, k, seed, outs[k])
        else:  # one call: k = 2 and k = 3 from the same staged inputs and discretisation
            mdfs.max_ig_multi(x, y, (2, 3), DIV, DISC, RANGE, XI, seed, out=outs)
            launches[0] += mdfs.last_launch_count()

    for w in range(args.warmup):
        step(100 + w)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    mdfs.profile(True)
    launches[0] = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step(1 + i)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = mdfs.profile_report()
    mdfs.profile(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    UNITS = _units()
    jobs = 1 if sharded else world  # one job split over the ranks, or one per rank
    value = jobs * UNITS * args.steps / total_s

    # ---- end to end through the C ABI with pinned host buffers ----
    x_h = torch.empty(ds.x.shape, dtype=torch.float32, pin_memory=True)
    x_h.copy_(torch.from_numpy(ds.x))
    y_h = torch.empty(ds.y.shape, dtype=torch.uint8, pin_memory=True)
    y_h.copy_(torch.from_numpy(ds.y))
    host_out = {k: (np.empty(M, np.float32), np.empty((M, max(k - 1, 1)), np.int32), np.empty(M, np.int32))
                for k in (2, 3)}
    def e2e_scan(k, seed):
        if sharded:  # host inputs in, merged keys decoded, results read back to the host
            res = scan(x_h, y_h, k, seed, None)
            for dst, src in zip(host_out[k], res):
                dst.reshape(-1)[:] = src.reshape(-1).cpu().numpy()
        else:
            mdfs.max_ig(x_h, y_h, k, DIV, DISC, RANGE, XI, seed, out=host_out[k])

    def e2e_step(seed):
        if sharded:
            for k in (2, 3):
                e2e_scan(k, seed)
        else:  # host buffers in and out of the one call
            mdfs.max_ig_multi(x_h, y_h, (2, 3), DIV, DISC, RANGE, XI, seed, out=host_out)

    e2e_step(99)
    e2e_t = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step(1 + i)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_t)
    if world > 1:
        t = torch.tensor([e2e_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    h2d = (2 if sharded else 1) * (x_h.numel() * 4 + y_h.numel())  # inputs staged once per call
    d2h = sum(a.nbytes for k in (2, 3) for a in host_out[k][: 1 + (k > 1)]) + sum(host_out[k][2].nbytes for k in (2, 3))

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel (k = 3 triple kernel) ----
    # Counting runs on the tensor cores as a one-hot E4M3 GEMM: the useful work
    # is one multiply-add per (triple, discretisation, sample) for the all-ones
    # voxel, 2 C(M,3) D N flops per launch.  The entropy epilogue skips the
    # table lookups of every triple that its SH3 lower bound rules out, so its
    # lookups are data-dependent and not the bound.  The peak is this GPU's
    # dense E4M3 rate measured in this run by the tcgen05 microbenchmark.
    peaks = peaks_run(local_rank) if not args.no_peaks else None
    roof = None
    k3 = prof.get("k3", None)
    if k3 and k3["count"]:
        avg_s = k3["ms"] / k3["count"] / 1e3
        evals = math.comb(M, 3) * DISC
        flops = 2.0 * evals * N_OBJ
        achieved = flops / avg_s / 1e12
        if peaks:
            peak, peak_src = peaks["fp8_mma_tflops"], "of measured (tcgen05 kind::f8f6f4 microbenchmark, this run)"
        else:
            bf16, bf16_src = _bf16_burst_peak()
            peak, peak_src = 2 * bf16, f"2 x {bf16_src} bf16 burst ({bf16} TF/s), of {bf16_src}"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k3tc_kernel", "launch_ms": 1e3 * avg_s,
                "per_launch": {"evals": evals, "useful_fp8_flop": flops},
                "peak_note": f"dense E4M3 {peak_src}",
                "traffic_note": "not measured in this run; DRAM bytes per launch from the ncu capture are in "
                                "profiles/ (the operand and pair records are read once: about 91 MB per launch)"}
    shares = {}
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    for kname, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        shares[kname] = {"launches": v["count"], "ms": round(v["ms"], 4), "share": round(v["ms"] / tot, 4)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "e4m3 one-hot MMA (f32 exact counts) + int32/int64 fixed-point entropy",
            "data": "synthetic",
            "config": _config({"parallelism": (f"one job's tuple tiles split over {world} GPUs, keys merged by "
                                               f"all-reduce MAX" if sharded else f"independent job per GPU x{world}")}),
            "step_ms_p50": float(np.percentile(step_ms, 50)), "step_ms_p99": float(np.percentile(step_ms, 99)),
            "wall_s_timed_region": wall,
            "gpu_launches": launches[0],
            "clocks": clk,
            "e2e": {"value": jobs * UNITS * args.steps / e2e_total, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "kernels": shares,
            # the stage count the library's tuner chose for this step's k = 2 launch
            "tuned": tuned_choices("k2tc_stages", M_VAR, N_OBJ, DIV + 1, DISC)}
    if args.serving_jobs > 0:
        line["serving"] = serving_run(args.serving_jobs, local_rank)
    if args.select_reps > 0:
        line["select"] = select_run(args.select_reps, local_rank)
    if args.interesting_reps > 0:
        line["interesting"] = interesting_run(args.interesting_reps, local_rank)
    if args.k4 and DIV == 1 and DISC * M_VAR ** 3 < 2**32:
        line["k4"] = k4_run(local_rank)
    if args.kgen:
        line["kgen"] = kgen_run(local_rank)
    if args.k5_m >= 5 and DIV == 1 and math.comb(args.k5_m, 4) < 2**32:
        line["k5"] = k5_run(args.k5_m, args.k5_disc, local_rank)
    if peaks:
        line["peaks"] = peaks
    if args.configs and not args.small:
        line["configs"] = configs_run(local_rank, args, peaks)
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        th = oracle.num_threads()
        n3 = max(1, th)  # one k = 3 variable per host thread
        nd = 15          # half of the discretisations: about 10-20 s of host work
        u, dt, th = oracle_sample(64, n3, n_disc=nd)
        line["cpu_baseline"] = {"value": u / dt, "unit": UNIT, "cores": th, "kind": "oracle",
                                "sample": f"64 variables at k=2 and {n3} at k=3, full partner scans over "
                                          f"{nd} of the {DISC} discretisations, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def peaks_run(device: int):
    """Measured rates of this GPU (library microbenchmarks): dense E4M3
    tcgen05 MMA throughput and random 4-byte shared-memory loads."""
    import torch
    from paper_1811_00631_gb300 import mdfs
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mma = mdfs.bench_mma_f8(40000)
    rnd = mdfs.bench_smem_lookup(4000, 0)
    win = mdfs.bench_smem_lookup(4000, 64)
    ghz = 2.07
    return {"fp8_mma_tflops": mma["tflops"], "fp8_mma_s": mma["seconds"],
            "smem_lookups_random_per_s": rnd["lookups_per_s"],
            "smem_lookups_window64_per_s": win["lookups_per_s"],
            "smem_lookups_random_per_sm_clock_at_2070mhz": rnd["lookups_per_s"] / sms / (ghz * 1e9),
            "smem_lookups_window64_per_sm_clock_at_2070mhz": win["lookups_per_s"] / sms / (ghz * 1e9),
            "how": "mdfs_bench_mma_f8 (one CTA per SM issuing tcgen05.mma kind::f8f6f4 128x256x32 on shared-memory "
                   "operands) and mdfs_bench_smem_lookup (8 xorshift index streams per thread over a 64 KB table, "
                   "whole table or 64-entry windows), CUDA events after a warm-up launch"}


def _parity(codes, y, c, k, xi, g_ig, g_tu, g_di, ref, variables):
    """Largest |IG - oracle| over the variables and how the argmax compares:
    equal, a different (d, S) that the tolerance rule allows (oracle's top two
    within 1e-4 + 1e-5 |o| and the GPU's choice within it of the maximum), or
    bad."""
    import oracle
    err, equal, allowed, bad = 0.0, 0, 0, 0
    for row, i in enumerate(variables):
        o = float(ref["ig"][row])
        tol = 1e-4 + 1e-5 * abs(o)
        err = max(err, abs(float(g_ig[i]) - o))
        S = [int(v) for v in g_tu[i]] if k > 1 else []
        if int(g_di[i]) == int(ref["disc"][row]) and (k == 1 or tuple(S) == tuple(int(v) for v in ref["tuples"][row])):
            equal += 1
            continue
        alt = oracle.ig_one(codes, y, c, xi, int(g_di[i]), int(i), S)
        if o - float(ref["second"][row]) <= tol and o - alt <= tol:
            allowed += 1
        else:
            bad += 1
    return {"max_abs_err": err, "argmax_equal": equal, "argmax_other_within_tol": allowed, "argmax_bad": bad,
            "variables": len(variables)}


def _time_scan(torch, fn, reps: int):
    """Median milliseconds of fn() over reps calls, CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def configs_run(device: int, args, peaks=None):
    """The other workloads of the method's configurations, each timed on the
    device and compared with the FP64 oracle on sampled variables (all of them
    for the small case):
      xor_N200_M50_k2:  200 x 50 XOR data, 2 classes, 1 discretisation;
      parity_N2000_M500_k1 / k2 (2 and 3 classes), 30 discretisations;
      parity_N2000_M500_k3: the bench step's k = 3 scan (two variables);
      batched_N1000_M20000_k2: 16 bootstrap folds x 4 label permutations in one
        call, 3 classes, 10 discretisations (spot check of three jobs, one job
        bit for bit against the single-job scan)."""
    import torch

    import oracle
    from paper_1811_00631_gb300 import mdfs, synth
    oracle.build()
    dev = torch.device("cuda", device)
    out = {}
    # XOR 200 x 50, k = 2 (latency-bound: one call is a few launches)
    ds = synth.xor_small()
    x, y = torch.from_numpy(ds.x).to(dev), torch.from_numpy(ds.y).to(dev)
    ms = _time_scan(torch, lambda: mdfs.max_ig(x, y, 2, 1, 1, 0.25, 0.25, 1), 20)
    g = [t.cpu().numpy() for t in mdfs.max_ig(x, y, 2, 1, 1, 0.25, 0.25, 1)]
    codes = oracle.discretize(ds.x, 1, 1, 0.25, 1)
    ref = oracle.max_ig(codes, ds.y, 2, 2, 0.25)
    out["xor_N200_M50_k2"] = {"ms_per_call": ms, "evals_per_s": math.comb(50, 2) / (ms / 1e3),
                              **_parity(codes, ds.y, 2, 2, 0.25, *g, ref, range(50))}
    # parity data 2000 x 500: k = 1, k = 2 with 2 and 3 classes, 30 discretisations
    ds = synth.madelon_like()
    x, y = torch.from_numpy(ds.x).to(dev), torch.from_numpy(ds.y).to(dev)
    rng = np.random.default_rng(3)
    noise = np.setdiff1d(np.arange(500), ds.informative)
    variables = np.concatenate([ds.informative, rng.choice(noise, 10, replace=False)]).astype(np.int32)
    for k, div in ((1, 1), (2, 1), (2, 2)):
        ms = _time_scan(torch, lambda: mdfs.max_ig(x, y, k, div, 30, 0.5, 0.25, 11), 5)
        g = [t.cpu().numpy() for t in mdfs.max_ig(x, y, k, div, 30, 0.5, 0.25, 11)]
        codes = oracle.discretize(ds.x, div, 30, 0.5, 11)
        ref = oracle.max_ig(codes, ds.y, div + 1, k, 0.25, variables=variables)
        out[f"parity_N2000_M500_k{k}_c{div + 1}"] = {
            "ms_per_call": ms, "evals_per_s": math.comb(500, k) * 30 / (ms / 1e3),
            **_parity(codes, ds.y, div + 1, k, 0.25, *g, ref, variables)}
    # k = 3 of the bench step: two variables, full partner scans over 30 discretisations
    g = [t.cpu().numpy() for t in mdfs.max_ig(x, y, 3, 1, 30, 0.5, 0.25, 11)]
    codes = oracle.discretize(ds.x, 1, 30, 0.5, 11)
    v3 = np.array([ds.info["base"][0], int(noise[0])], dtype=np.int32)
    ref = oracle.max_ig(codes, ds.y, 2, 3, 0.25, variables=v3)
    out["parity_N2000_M500_k3_c2"] = {"timing": "the bench step's k = 3 launch (roofline)",
                                      **_parity(codes, ds.y, 2, 3, 0.25, *g, ref, v3)}
    if args.batch_configs:
        out["batched_N1000_M20000_k2_c3"] = batched_check(device, args.batch_folds, args.batch_perms, args.batch_m,
                                                           peaks)
    return out


def k2_roofline(pair_discs: float, N: int, c: int, k2: dict, peaks: dict) -> dict:
    """Roofline entry of the k = 2 tensor-core kernel: algorithmic work 2 c^2 N
    FLOP per (pair, discretisation) (every voxel count an N-term dot product of
    bin indicators), and beside it the work of the products the kernel forms on
    the tensor cores, 2 (c - 1)^2 N (the bins >= 1; the other voxels follow from
    the margins)."""
    secs = k2["ms"] / 1e3
    useful = pair_discs * 2.0 * c * c * N
    formed = pair_discs * 2.0 * (c - 1) * (c - 1) * N
    peak = peaks["fp8_mma_tflops"]
    return {"bound": "tensor", "kernel": "k2tc3_kernel" if c == 3 else "k2tc_kernel", "launches": k2["count"],
            "kernel_s": secs, "achieved": useful / secs / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": useful / secs / 1e12 / peak, "algorithmic_flop": useful,
            "formed_tflops": formed / secs / 1e12, "formed_frac": formed / secs / 1e12 / peak,
            "unit_note": "2 c^2 N FLOP per (pair, discretisation); formed_*: the 2 (c-1)^2 N the MMAs compute",
            "peak_note": "dense E4M3 of measured (tcgen05 kind::f8f6f4 microbenchmark, this run)"}


def batched_check(device: int, n_folds: int, n_perms: int, M: int, peaks=None):
    """The batched workload in one mdfs_max_ig_batch call, timed with CUDA
    events; three jobs spot-checked against the oracle and one job bit for bit
    against the single-job scan of its resampled data."""
    import torch

    import oracle
    from paper_1811_00631_gb300 import mdfs, synth
    dev = torch.device("cuda", device)
    N, D, div, r, xi, seed = 1000, 10, 2, 0.5, 0.25, 1
    ds = synth.xor_pairs(N=N, M=M, n_pairs=100, seed=4)
    idx, yperm = synth.bootstrap_jobs(N, n_folds=n_folds, n_perms=n_perms, seed=5)
    si = np.repeat(idx, n_perms, axis=0).astype(np.int32)
    yp = np.tile(yperm, (n_folds, 1)).astype(np.int32)
    x, y = torch.from_numpy(ds.x).to(dev), torch.from_numpy(ds.y).to(dev)
    sid, ypd = torch.from_numpy(si).to(dev), torch.from_numpy(yp).to(dev)
    J = n_folds * n_perms
    mdfs.max_ig_batch(x, y, sid[:1], ypd[:1], n_jobs=1, k=2, divisions=div, discretizations=D, range_=r, seed=seed)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mdfs.profile(True)  # per-launch CUDA events, no synchronisation
    a.record()
    ig, tu, di = mdfs.max_ig_batch(x, y, sid, ypd, n_jobs=J, k=2, divisions=div, discretizations=D, range_=r,
                                   pc_xi=xi, seed=seed)
    b.record()
    b.synchronize()
    prof = mdfs.profile_report()
    mdfs.profile(False)
    secs = a.elapsed_time(b) / 1e3
    ig, tu, di = ig.cpu().numpy(), tu.cpu().numpy(), di.cpu().numpy()
    pairs = ds.info["pairs"]
    found = sum(int(tu[0, p, 0] == q) + int(tu[0, q, 0] == p) for p, q in pairs)
    rng = np.random.default_rng(17)
    checks = []
    for j in (0, J // 2, J - 1):
        xj = np.ascontiguousarray(ds.x[:, si[j]])
        yj = ds.y[yp[j][si[j]]]
        codes = oracle.discretize(xj, div, D, r, seed)
        p, q = pairs[rng.integers(len(pairs))]
        variables = np.array(sorted({int(p), int(q), *rng.choice(M, 2, replace=False).tolist()}), np.int32)
        ref = oracle.max_ig(codes, yj, div + 1, 2, xi, variables=variables)
        checks.append(_parity(codes, yj, div + 1, 2, xi, ig[j], tu[j], di[j], ref, variables))
    j = J - 1
    w = mdfs.max_ig(torch.from_numpy(np.ascontiguousarray(ds.x[:, si[j]])).to(dev),
                    torch.from_numpy(ds.y[yp[j][si[j]]]).to(dev), 2, div, D, r, xi, seed)
    single_equal = all(np.array_equal(u, v.cpu().numpy()) for u, v in zip((ig[j], tu[j], di[j]), w))
    # the tensor-core k = 2 kernel against the measured E4M3 rate, in the
    # algorithmic unit of the one-hot formulation: every voxel's class count
    # is an N-term dot product of bin indicators, 2 c^2 N FLOP per (pair,
    # discretisation); the kernel forms the 2 x 2 block of bins >= 1 on the
    # tensor cores (2 (c - 1)^2 N) and derives the other voxels from margins
    k2 = prof.get("k2", {"count": 0, "ms": 0.0})
    roof = None
    if peaks and k2["ms"] > 0:
        roof = k2_roofline(J * math.comb(M, 2) * D, N, div + 1, k2, peaks)
    return {"jobs": J, "seconds": secs, "evals_per_s": J * math.comb(M, 2) * D / secs, "roofline": roof,
            "kernels": prof, "tuned": tuned_choices("k2tc_batch_stages", M, N, div + 1, D),
            "max_abs_err": max(c["max_abs_err"] for c in checks),
            "argmax_bad": sum(c["argmax_bad"] for c in checks),
            "argmax_equal": sum(c["argmax_equal"] for c in checks),
            "argmax_other_within_tol": sum(c["argmax_other_within_tol"] for c in checks),
            "variables_checked": sum(c["variables"] for c in checks),
            "job_equals_single_job_scan": bool(single_equal),
            "xor_partners_recovered_job0": f"{found}/{2 * len(pairs)}"}


def select_run(reps: int, device: int):
    """The canonical selection pipeline (contrasts, IG scan over the extended
    set, fit on the contrasts, Holm-adjusted p-values, relevant set) on 2000 x
    500 data with 5 planted XOR pairs (10% label flips; a pair is invisible to
    single-variable tests) and n_contrast = M = 500, for k = 2 and k = 3.
    Timed with CUDA events on the current stream around whole mdfs_select
    calls (device-resident inputs; the call returns after the result is on the
    device).  evals counts unordered tuples of the extended set x
    discretisations."""
    import torch
    from paper_1811_00631_gb300 import mdfs, synth
    dev = torch.device("cuda", device)
    ds = synth.xor_pairs(N=N_OBJ, M=M_VAR, n_pairs=5, flip=0.1, seed=4)
    x = torch.from_numpy(ds.x).to(dev)
    y = torch.from_numpy(ds.y).to(dev)
    nc = M_VAR
    out = {"workload": f"xor-pairs data N={N_OBJ} M={M_VAR} (5 planted pairs) + {nc} contrast variables, "
                       f"D={DISC}, c={DIV + 1}, Holm at 0.05"}
    for k in (2, 3):
        r = mdfs.select(x, y, nc, k, DIV, DISC, RANGE, XI, seed=5)  # warm-up
        stream = torch.cuda.current_stream(dev)
        ts = []
        for i in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = mdfs.select(x, y, nc, k, DIV, DISC, RANGE, XI, seed=5 + i)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        evals = math.comb(M_VAR + nc, k) * DISC
        rel = r["relevant"].cpu().numpy()
        out[f"k{k}"] = {"ms": ms, "evals_per_s": evals / (ms / 1e3), "selected": int(rel.sum()),
                        "informative_selected": int(rel[ds.informative].sum()),
                        "informative": int(len(ds.informative)), "ig_lim": r["ig_lim"], "n_eff": r["n_eff"]}
    return out


def interesting_run(reps: int, device: int):
    """Interesting tuples (every (variable, partner set) whose IG, maximised
    over the discretisations, reaches a threshold) on the bench data (2000 x
    500, 30 discretisations, 2 classes) at k = 2 and k = 3, timed with CUDA
    events around whole mdfs_interesting_tuples calls with device-resident
    inputs.  The threshold is the 90th percentile of the variables' IG^k_max
    (one untimed max scan), so the informative variables' strong tuples
    qualify.  evals counts unordered tuples x discretisations."""
    import torch
    from paper_1811_00631_gb300 import mdfs, synth
    dev = torch.device("cuda", device)
    ds = synth.madelon_like(N=N_OBJ, M=M_VAR, seed=2)
    x = torch.from_numpy(ds.x).to(dev)
    y = torch.from_numpy(ds.y).to(dev)
    out = {"workload": f"parity data N={N_OBJ} M={M_VAR}, D={DISC}, c={DIV + 1}; threshold = 90th percentile "
                       f"of IG^k_max"}
    for k in (2, 3):
        best, _, _ = mdfs.max_ig(x, y, k, DIV, DISC, RANGE, XI, 7)
        thr = float(np.quantile(best.cpu().numpy(), 0.9))
        cap = 1 << 20
        got = mdfs.interesting_tuples(x, y, k, DIV, DISC, RANGE, XI, 7, thr, capacity=cap)  # warm-up
        stream = torch.cuda.current_stream(dev)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            got = mdfs.interesting_tuples(x, y, k, DIV, DISC, RANGE, XI, 7, thr, capacity=cap)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        evals = math.comb(M_VAR, k) * DISC
        out[f"k{k}"] = {"ms": ms, "evals_per_s": evals / (ms / 1e3), "threshold": thr, "records": int(len(got[0]))}
    return out


def kgen_run(device: int):
    """k = 4 and k = 5 with three classes per variable (divisions = 2: every
    voxel of every tuple counted from the bit planes) on madelon-shaped data
    with N = 2000: k = 4 on M = 120 variables and 10 discretisations, k = 5 on
    M = 48 and 2, each timed with CUDA events after a one-discretisation
    warm-up.  evals counts unordered tuples x discretisations."""
    import torch
    from paper_1811_00631_gb300 import mdfs, synth
    dev = torch.device("cuda", device)
    out = {"workload": f"madelon-shaped parity data N={N_OBJ}, c=3 (divisions 2)"}
    stream = torch.cuda.current_stream(dev)
    for k, m, nd in ((4, 120, 10), (5, 48, 2)):
        ds = synth.madelon_like(N=N_OBJ, M=m, seed=2)
        x = torch.from_numpy(ds.x).to(dev)
        y = torch.from_numpy(ds.y).to(dev)
        mdfs.max_ig(x, y, k, 2, 1, RANGE, XI, 1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mdfs.max_ig(x, y, k, 2, nd, RANGE, XI, 5)
        b.record(stream)
        b.synchronize()
        sec = a.elapsed_time(b) / 1e3
        evals = math.comb(m, k) * nd
        out[f"k{k}"] = {"M": m, "discretizations": nd, "s": sec, "evals_per_s": evals / sec,
                        "voxels_per_tuple": 3 ** k}
    return out


def k4_run(device: int):
    """One k = 4 scan of the bench data (2000 x 500, 30 discretisations, 2
    classes): C(500, 4) x 30 = 7.7e10 quadruple x discretisation evaluations,
    timed with CUDA events after a one-discretisation warm-up."""
    import torch
    from paper_1811_00631_gb300 import mdfs, synth
    dev = torch.device("cuda", device)
    ds = synth.madelon_like(M=M_VAR, seed=2)
    x = torch.from_numpy(ds.x).to(dev)
    y = torch.from_numpy(ds.y).to(dev)
    mdfs.max_ig(x, y, 4, DIV, 1, RANGE, XI, 1)
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    mdfs.max_ig(x, y, 4, DIV, DISC, RANGE, XI, 5)
    b.record(stream)
    b.synchronize()
    s = a.elapsed_time(b) / 1e3
    evals = math.comb(M_VAR, 4) * DISC
    return {"workload": f"madelon-shaped parity data N={N_OBJ} M={M_VAR}, k=4, D={DISC}, c={DIV + 1}",
            "s": s, "evals_per_s": evals / s,
            "paper_context": "Table 2 of the paper: 4D, 30 discretisations, Madelon 2000 x 500 on a Tesla K80: 456 s"}


def k5_run(m: int, n_disc: int, device: int):
    """One k = 5 scan with n_disc discretisations of the bench data's
    generator with m variables (madelon-shaped, 2000 samples, 2 classes):
    C(m, 5) x n_disc quintuple evaluations, timed with CUDA events after a
    warm-up on a 40-variable subset."""
    import torch
    from paper_1811_00631_gb300 import mdfs, synth
    dev = torch.device("cuda", device)
    ds = synth.madelon_like(M=m, seed=2)
    x = torch.from_numpy(ds.x).to(dev)
    y = torch.from_numpy(ds.y).to(dev)
    mdfs.max_ig(x[:40].contiguous(), y, 5, DIV, 1, RANGE, XI, 1)
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    mdfs.max_ig(x, y, 5, DIV, n_disc, RANGE, XI, 5)
    b.record(stream)
    b.synchronize()
    s = a.elapsed_time(b) / 1e3
    evals = math.comb(m, 5) * n_disc
    return {"workload": f"madelon-shaped parity data N={N_OBJ} M={m}, k=5, D={n_disc}, c={DIV + 1}",
            "s": s, "evals_per_s": evals / s,
            "paper_context": "Madelon 2000 x 500 at 5D on the paper's GPU: 1 h with 1 discretisation (Table 1), "
                             "42 h with 30 (Table 2)"}


def serving_run(n_jobs: int, device: int):
    """Serving-mix measurement: a closed-loop pass measures capacity (jobs/s),
    then a Poisson stream at 70% of that capacity gives the job latencies."""
    from paper_1811_00631_gb300 import serve, synth
    specs = synth.serving_mix(n_jobs=n_jobs, seed=17, rate_hz=1.0, n_range=(100, 5000), m_range=(100, 5000),
                              max_work=2e10)
    jobs = []
    evals = 0.0
    for sp in specs:
        x, y = synth.serving_data(sp)
        jobs.append(serve.Job(x=x, y=y, k=sp["k"], divisions=sp["divisions"], discretizations=sp["discretizations"],
                              range_=0.5, pc_xi=0.25, seed=sp["seed"], alpha=0.05, tag=sp["job"]))
        evals += serve.job_evals(sp["M"], sp["k"], sp["discretizations"])
    with serve.Server(n_slots=4, device=device) as srv:  # warm-up: workspaces and modules
        for f in [srv.submit(j) for j in jobs[:8]]:
            f.result()
        busy = BusySampler(device)
        busy.start()
        t0 = time.perf_counter()
        for f in [srv.submit(j) for j in jobs]:
            f.result()
        closed_s = time.perf_counter() - t0
        busy_closed = busy.stop()
        capacity = n_jobs / closed_s
        rate = 0.7 * capacity
        rng = np.random.default_rng(3)
        gaps = rng.exponential(1.0 / rate, size=n_jobs)
        busy = BusySampler(device)
        busy.start()
        t0 = time.perf_counter()
        futs = []
        for j, g in zip(jobs, np.cumsum(gaps)):
            delay = g - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(j))
        results = [f.result() for f in futs]
        open_s = time.perf_counter() - t0
        busy_open = busy.stop()
    st = serve.latency_stats(results)
    return {"jobs": n_jobs, "slots": 4, "capacity_jobs_per_s": capacity, "arrival_rate_jobs_per_s": rate,
            "p50_ms": 1e3 * st["p50_s"], "p99_ms": 1e3 * st["p99_s"], "mean_ms": 1e3 * st["mean_s"],
            "evals_per_s_closed_loop": evals / closed_s, "evals_per_s_poisson": evals / open_s,
            "gpu_busy_closed_loop": busy_closed, "gpu_busy_poisson": busy_open,
            "staging": "pinned per-slot input buffers, one packed result read per job",
            "mix": "k in 1..3, N U[100,5000], M log-U[100,5000] capped at C(M,k)*D*N <= 2e10, f32/i8, "
                   "divisions 1-3, 5-30 discretisations, each scan followed by the IG_lim fit"}


def run_batched(args):
    """Batched k = 2 workload: N = 1000 x M = 20000 (100 XOR pairs), 3 classes,
    10 discretisations, bootstrap folds x y-permutations in one batched call."""
    import torch

    from paper_1811_00631_gb300 import build, mdfs, synth
    build.build()
    n_folds, n_perms = args.batch_folds, args.batch_perms
    N, M, D, div = 1000, args.batch_m, 10, 2
    ds = synth.xor_pairs(N=N, M=M, n_pairs=100, seed=4)
    idx, yperm = synth.bootstrap_jobs(N, n_folds=n_folds, n_perms=n_perms, seed=5)
    si = torch.from_numpy(np.repeat(idx, n_perms, axis=0).astype(np.int32)).cuda()
    yp = torch.from_numpy(np.tile(yperm, (n_folds, 1)).astype(np.int32)).cuda()
    x = torch.from_numpy(ds.x).cuda()
    y = torch.from_numpy(ds.y).cuda()
    J = n_folds * n_perms
    mdfs.max_ig_batch(x, y, si[:1], yp[:1], n_jobs=1, k=2, divisions=div, discretizations=D, range_=0.5, seed=1)
    torch.cuda.synchronize()
    mdfs.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    ig, tu, di = mdfs.max_ig_batch(x, y, si, yp, n_jobs=J, k=2, divisions=div, discretizations=D, range_=0.5,
                                   seed=1)
    ev1.record()
    torch.cuda.synchronize()
    prof = mdfs.profile_report()
    mdfs.profile(False)
    secs = ev0.elapsed_time(ev1) / 1e3
    evals = J * math.comb(M, 2) * D
    found = 0
    pairs = ds.info["pairs"]
    ig0, tu0 = ig[0].cpu().numpy(), tu[0].cpu().numpy()
    for a, b in pairs:
        found += int(tu0[a, 0] == b) + int(tu0[b, 0] == a)
    roof = None
    if not args.no_peaks and prof.get("k2", {}).get("ms"):
        roof = k2_roofline(J * math.comb(M, 2) * D, N, div + 1, prof["k2"], peaks_run(0))
    line = {"metric": "batched k=2 tuple*disc evals/sec", "value": evals / secs, "unit": UNIT, "n_gpus": 1,
            "jobs": J, "seconds": secs, "config": {"N": N, "M": M, "divisions": div, "discretizations": D,
                                                   "folds": n_folds, "perms": n_perms},
            "roofline": roof, "kernels": {k: v for k, v in prof.items()},
            "tuned": tuned_choices("k2tc_batch_stages", M, N, div + 1, D),
            "xor_partners_recovered_job0": f"{found}/{2 * len(pairs)}"}
    print(json.dumps(line), flush=True)
    return 0


def tuned_choices(kernel: str, M: int, N: int, c: int, D: int):
    """The library's cached launch choice for a shape, read back from its
    MDFS_TUNE_FILE ("<kernel> M=.. N=.. c=.. D=.. -> <choice>" lines); None
    when the file is unset or holds no entry."""
    path = os.environ.get("MDFS_TUNE_FILE")
    if not path or not os.path.exists(path):
        return None
    key = f"{kernel} M={M} N={N} c={c} D={D} -> "
    vals = [ln.split(" -> ")[1].strip() for ln in open(path) if ln.startswith(key)]
    return {"key": key[:-4], "stages": int(vals[-1])} if vals else None


def _tune_file_for_this_run():
    """A fresh tuning cache per bench process (so the line names what this run
    chose), unless the caller set one."""
    if "MDFS_TUNE_FILE" not in os.environ:
        log_dir = os.environ.get("MDFS_BENCH_LOG_DIR") or tempfile.gettempdir()
        path = os.path.join(log_dir, f"mdfs_tune_{os.getpid()}.txt")
        if os.path.exists(path):
            os.remove(path)
        os.environ["MDFS_TUNE_FILE"] = path


def main():
    _tune_file_for_this_run()
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="reduced profiling case (M=500, D=--small-disc)")
    ap.add_argument("--small-disc", type=int, default=2, help="discretisations of the --small case")
    ap.add_argument("--serving-jobs", type=int, default=512, help="jobs of the serving-mix run (0: skip)")
    ap.add_argument("--k4", type=int, default=1, help="time one k = 4 scan of the bench data (0: skip)")
    ap.add_argument("--kgen", type=int, default=1,
                    help="time the k = 4 and k = 5 scans with three classes per variable (0: skip)")
    ap.add_argument("--k5-m", type=int, default=200,
                    help="variables of the timed one-discretisation k = 5 scan (0: skip; 500 = the "
                         "madelon-shaped 5D case, about 19 s per discretisation)")
    ap.add_argument("--k5-disc", type=int, default=1, help="discretisations of the timed k = 5 scan")
    ap.add_argument("--select-reps", type=int, default=3,
                    help="timed calls of the selection pipeline per k (0: skip)")
    ap.add_argument("--interesting-reps", type=int, default=3,
                    help="timed interesting-tuple calls per k on the bench data (0: skip)")
    ap.add_argument("--shard", action="store_true",
                    help="split one job's tuple space over the ranks (the default with more than one GPU)")
    ap.add_argument("--independent", action="store_true",
                    help="with more than one GPU, run an independent job per rank instead (weak scaling)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the tensor-core and shared-memory microbenchmarks")
    ap.add_argument("--configs", type=int, default=1, help="time the other configurations with oracle checks (0: skip)")
    ap.add_argument("--batch-configs", type=int, default=1,
                    help="include the batched 64-job workload among the configurations (0: skip)")
    ap.add_argument("--batched", action="store_true", help="run the batched k=2 workload instead")
    ap.add_argument("--batch-folds", type=int, default=16)
    ap.add_argument("--batch-perms", type=int, default=4)
    ap.add_argument("--batch-m", type=int, default=20000)
    args = ap.parse_args()
    if args.small:
        _use_small_case(args.small_disc)
        args.configs = 0
        args.serving_jobs = 0
        args.select_reps = 0
        args.interesting_reps = 0
        args.kgen = 0
        args.k4 = 0
        args.k5_m = 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.batched:
        return run_batched(args)
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return 0
        return run_reference(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    try:
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark: S = A R and S' = A^T R throughput on GB300 (GB/s of A).

One step is one pass of the whole sketching path over the n = 32768 FP32
kernel-matrix workload (A_ij = exp(-||x_i - y_j||^2 / (2 * 0.1^2)), X != Y,
32768 points each, uniform in [0,1]^3; A resident in HBM, 4.29 GB):

  1. operator generation: block SJLT (d = 256, alpha = 4), SRHT (d = 256),
     Gaussian (d = 256);
  2. S and S' for each operator (SJLT on CUDA cores in FP32; SRHT and
     Gaussian on the fastest available path);
  3. the adaptive SJLT run: d0 = 128, Delta-d = 64, up to 512 columns, stopping
     test after every increment (eps_rel = 1e-2, eps_abs = 1e-8), S and S'.

value = bytes of A streamed by all sketch products of the step / step time.
A is larger than L2 (126 MB), so no flush is needed between steps.

The same line carries, measured in the same run on rank 0 at N = 1 (skip with
--no-extra), the precision comparison (key "precision": the Gaussian S = A R
of the 65536 x 65536 FP32 kernel matrix at d = 512 on FP32 CUDA cores, as a
bf16 hi+lo split and in scaled FP8 on the tensor cores, each error on 4096
sampled rows), the differentiation workload (key "differentiation": the
matrix-free S = K(X, X; h) R of 262144 points and its adjoint, against the
explicit-K path, with their ALU rooflines and the FP64 oracle gradient timed
on a 4096-point problem as their CPU baseline) and the per-node adaptive loop
of Algorithm 1 (key "hss": the n = 2048 FP64 kernel matrix, leaf 64, whole
compressions, with the FP64 oracle's time as its CPU baseline).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.  Under torchrun every rank runs an independent
replica (the path is not sharded); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "S=A·R throughput (GB/s of A, % HBM peak) per JL operator at stated error"
WORKLOAD = dict(name="kernel_fp32_n32768", n=32768, d=256, alpha=4, h=0.1, seed=20230203 + 1,
                d0=128, dd=64, d_max=512, eps_rel=1e-2, eps_abs=1e-8)


# ---------------------------------------------------------------------------
# Multi-rank bookkeeping (N independent replicas, one per GPU): the job's time
# is the slowest rank's, and the job's value counts every rank's work.
def reduce_time_max(elapsed: float, world: int, device) -> float:
    """Max of `elapsed` over the ranks of the default process group (NCCL on
    the GPUs, gloo on CPU); `elapsed` itself when world == 1."""
    if world <= 1:
        return float(elapsed)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_pass: float, passes_per_rank: int, world: int, elapsed: float) -> float:
    """GB/s of A for the whole job: all ranks' passes over their A / the job's time."""
    return bytes_per_pass * passes_per_rank * world / elapsed / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
class Step:
    """Everything one step does, with per-call CUDA events."""

    def __init__(self, A, n, prec_dense, timed_events=True, only="all"):
        import torch
        from paper_2302_01977_gb300 import jlsketch as jl
        self.jl, self.torch = jl, torch
        self.A, self.n = A, n
        self.prec_dense = prec_dense
        w = WORKLOAD
        dev = A.device
        self.bufs = {k: torch.empty((n, w["d"]), dtype=torch.float32, device=dev)
                     for k in ("sjlt_S", "sjlt_St", "srht_S", "srht_St", "gauss_S", "gauss_St")}
        self.adS = torch.empty((n, w["d_max"]), dtype=torch.float32, device=dev)
        self.adSt = torch.empty((n, w["d_max"]), dtype=torch.float32, device=dev)
        self.events = []  # (label, start, end)
        self.timed = timed_events
        self.only = only
        self.adaptive_info = None

    def _ev(self, label, fn):
        if not self.timed:
            fn()
            return
        s = self.torch.cuda.Event(enable_timing=True)
        e = self.torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        self.events.append((label, s, e))

    def run(self, step_idx):
        jl, A, w = self.jl, self.A, WORKLOAD
        seed = w["seed"] + 7919 * step_idx
        hs = []
        try:
            ops = [("sjlt", "sjlt_block", w["alpha"], self.prec_dense),
                   ("srht", "srht", 1, self.prec_dense), ("gauss", "gauss", 1, self.prec_dense)]
            passes = 0
            for name, kind, alpha, prec in ops:
                if self.only not in ("all", name):
                    continue
                passes += 2
                h = jl.sketch_create(kind, self.n, w["d"], alpha, seed, w["d"])
                hs.append(h)
                S, St = self.bufs[name + "_S"], self.bufs[name + "_St"]
                self._ev(f"{name}.S", lambda: jl.sketch_apply(h, A, jl.SK_S, prec, S=S))
                self._ev(f"{name}.St", lambda: jl.sketch_apply(h, A, jl.SK_ST, prec, St=St))
            if self.only not in ("all", "adaptive"):
                return passes
            # adaptive SJLT run (Algorithm 1 on the global sketch)
            h = jl.sketch_create("sjlt_block", self.n, w["d0"] + w["dd"], w["alpha"], seed + 1, w["d_max"])
            hs.append(h)
            self._ev("adaptive.apply",
                     lambda: jl.sketch_apply(h, A, jl.SK_BOTH, self.prec_dense, S=self.adS, St=self.adSt))
            d, hist = w["d0"], []
            passes += 2
            ad_passes = 2
            while True:
                wd = d + w["dd"]
                s1, s2 = jl.adaptive_norm_test_pair(h, self.adS[:, :wd], self.adSt[:, :wd], w["dd"], w["eps_rel"],
                                                    w["eps_abs"])
                hist.append((d, s1[1] / s1[2], s2[1] / s2[2]))
                if (s1[0] and s2[0]) or wd + w["dd"] > w["d_max"]:
                    converged = s1[0] and s2[0]
                    break
                jl.sketch_increment(h, w["dd"])
                self._ev("adaptive.increment",
                         lambda: jl.sketch_apply_increment(h, A, jl.SK_BOTH, self.prec_dense, S=self.adS,
                                                           St=self.adSt))
                passes += 2
                ad_passes += 2
                d += w["dd"]
            self.adaptive_info = dict(d_reached=d + w["dd"], converged=bool(converged), passes_over_A=ad_passes,
                                      ratios=[(int(a), round(b, 6), round(c, 6)) for a, b, c in hist])
            return passes  # passes over A in this step
        finally:
            for h in hs:
                jl.sketch_destroy(h)


def kernel_times(events):
    """label -> list of ms."""
    out = {}
    for label, s, e in events:
        out.setdefault(label, []).append(s.elapsed_time(e))
    return out


# ---------------------------------------------------------------------------
def cpu_baseline(X, Y, S_gpu, rows_per_product, seed):
    """Time the FP64 oracle on a bounded sample and check the GPU results on it."""
    import numpy as np

    from oracle import operators as ops
    from oracle import sketch as osk
    w = WORKLOAD
    n, d = w["n"], w["d"]
    rng = np.random.default_rng(12345)
    rows = np.sort(rng.choice(n, rows_per_product, replace=False))
    A_rows = osk.kernel_matrix(X[rows], Y, w["h"])          # inputs prepared before timing
    A_cols = osk.kernel_matrix(X, Y[rows], w["h"]).T
    t0 = time.perf_counter()
    errs = {}
    for name, kind, alpha in (("sjlt", "sjlt_block", w["alpha"]), ("srht", "srht", 1), ("gauss", "gauss", 1)):
        R = ops.Operator(kind, n, d, alpha, seed).dense()
        S_s = A_rows @ R
        St_s = A_cols @ R
        if S_gpu is not None:
            gs, gst = S_gpu[name]
            errs[name] = max(float(np.linalg.norm(gs[rows] - S_s) / np.linalg.norm(S_s)),
                             float(np.linalg.norm(gst[rows] - St_s) / np.linalg.norm(St_s)))
    dt = time.perf_counter() - t0
    bytes_a = 6 * rows_per_product * n * 4
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return dict(value=bytes_a / dt / 1e9, unit="GB/s", cores=cores, kind="oracle",
                sample=f"{rows_per_product} sampled rows of S and of S' for each of SJLT, SRHT, Gaussian "
                       f"(operators formed densely in FP64, products by numpy), {dt:.1f} s",
                seconds=dt), errs


def traffic_from_profile(kernel_file, record="sjlt_traffic.json.txt"):
    """dram bytes per launch recorded in profiles/ for the current source, else None."""
    p = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(p):
        return None
    try:
        rec = json.loads(open(p).read())
    except ValueError:
        return None
    src = os.path.join(ROOT, "paper_2302_01977_gb300", "csrc", kernel_file)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    return rec


# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = WORKLOAD
    n = w["n"] = args.n
    w["name"] = f"kernel_fp32_n{n}"
    X = inputs.points(n, seed=w["seed"])
    Y = inputs.points(n, seed=w["seed"] + 1000)
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    jl.kernel_matrix(jl.generator(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), w["h"]), A)
    prec_dense = jl.SK_PREC_BF16X2 if args.prec == "bf16x2" else jl.SK_PREC_NATIVE
    if args.prec == "auto":
        prec_dense = jl.SK_PREC_NATIVE
        try:  # use the tensor-core path when the library provides it
            h = jl.sketch_create("gauss", 1024, 64, 1, 1, 64)
            T = torch.zeros((1024, 1024), device="cuda")
            O = torch.zeros((1024, 64), device="cuda")
            jl.sketch_apply(h, T, jl.SK_S, jl.SK_PREC_BF16X2, S=O)
            jl.sketch_destroy(h)
            prec_dense = jl.SK_PREC_BF16X2
        except jl.JLSketchError:
            pass
    step = Step(A, n, prec_dense, only=args.only)
    for i in range(args.warmup):
        step.run(i)
    torch.cuda.synchronize()
    step.events.clear()
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = jl.sketch_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    passes = 0
    for i in range(args.steps):
        passes += step.run(args.warmup + i)
    t_end.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = jl.sketch_launch_count() - launches0
    clk = clocks.stop()
    elapsed = reduce_time_max(t_start.elapsed_time(t_end) / 1e3, world, "cuda")
    bytes_a = n * n * 4
    value = job_value(bytes_a, passes, world, elapsed)
    times = kernel_times(step.events)
    hbm, bf16, bf16s, peak_kind = peaks()

    per_op = {}
    for name in ("sjlt", "srht", "gauss"):
        if f"{name}.S" not in times:
            continue
        ts, tst = statistics.median(times[f"{name}.S"]), statistics.median(times[f"{name}.St"])
        per_op[name] = {"S_gbs": round(bytes_a / ts / 1e6, 1), "St_gbs": round(bytes_a / tst / 1e6, 1),
                        "S_ms": round(ts, 4), "St_ms": round(tst, 4),
                        "pct_hbm_S": round(100 * bytes_a / ts / 1e6 / hbm, 1),
                        "pct_hbm_St": round(100 * bytes_a / tst / 1e6 / hbm, 1)}
    for name in ("srht", "gauss"):
        if name in per_op:
            per_op[name]["prec"] = "bf16x2" if prec_dense == jl.SK_PREC_BF16X2 else "fp32"
    sjlt_routes = {"S": -1, "St": -1}
    if "sjlt" in per_op:
        if prec_dense == jl.SK_PREC_BF16X2:  # each product's route, picked by timing on its first call
            sjlt_routes = {"S": jl.sketch_sjlt_route("sjlt_block", n, n, n, w["d"], jl.SK_S),
                           "St": jl.sketch_sjlt_route("sjlt_block", n, n, n, w["d"], jl.SK_ST)}
        per_op["sjlt"]["prec"] = "bf16x2 allowed" if prec_dense == jl.SK_PREC_BF16X2 else "fp32"
        per_op["sjlt"]["route"] = {k: {1: "tensor-core +-1 product", 0: "SJLT kernel", -1: "SJLT kernel"}[v]
                                   for k, v in sjlt_routes.items()}
    if step.adaptive_info:
        per_op["adaptive_sjlt"] = dict(step.adaptive_info)

    # dominant kernel: the class with the largest total time in the timed region
    totals = {k: sum(v) for k, v in times.items()}
    cls = {"sjlt_rows": totals.get("sjlt.S", 0), "sjlt_cols": totals.get("sjlt.St", 0),
           "srht": totals.get("srht.S", 0) + totals.get("srht.St", 0),
           "gauss": totals.get("gauss.S", 0) + totals.get("gauss.St", 0)}
    # where the step's time goes: the sketch products by operator, the adaptive run's sketches
    # (S and S' of its first sketch and increments), and the rest (stopping tests, host)
    step_ms = 1e3 * elapsed / args.steps
    sketched = {"sjlt": cls["sjlt_rows"] + cls["sjlt_cols"], "srht": cls["srht"], "gauss": cls["gauss"],
                "adaptive_sketches": totals.get("adaptive.apply", 0) + totals.get("adaptive.increment", 0)}
    per_step = {k: v / args.steps for k, v in sketched.items()}
    per_step["stopping_tests_and_host"] = max(0.0, step_ms - sum(per_step.values()))
    step_share = {k: round(v / step_ms, 3) for k, v in per_step.items()}
    d_out_bytes = n * w["d"] * 4
    ccs_bytes = n * w["alpha"] * 2 + (n // 512) * (w["d"] + 4) * 4
    # the SJLT kernels are the ones the roofline tracks (HBM-bound, one pass of A)
    sj = "sjlt_cols" if cls["sjlt_cols"] >= cls["sjlt_rows"] else "sjlt_rows"
    key = "sjlt.St" if sj == "sjlt_cols" else "sjlt.S"
    t_launch = statistics.median(times[key]) / 1e3 if key in times else float("inf")
    alg_bytes = bytes_a + d_out_bytes + ccs_bytes
    achieved = alg_bytes / t_launch / 1e9
    prof = traffic_from_profile("sjlt_apply.cu")
    traffic = None
    if prof:
        traffic = prof.get("cols_bytes_per_launch" if sj == "sjlt_cols" else "rows_bytes_per_launch")
    tc_route = sjlt_routes["St" if sj == "sjlt_cols" else "S"] == 1
    if tc_route:
        kname = "tc_sketch_kernel (SJLT " + ("S' = A^T R" if sj == "sjlt_cols" else "S = A R") + ", +-1 product)"
        tcp = traffic_from_profile("gemm_tc.cu", "tc_traffic.json.txt")  # the tensor-core kernel's counters
        traffic = tcp.get("cols_bytes_per_launch" if sj == "sjlt_cols" else "rows_bytes_per_launch") if tcp else None
    else:
        kname = "sjlt_cols_kernel (S' = A^T R)" if sj == "sjlt_cols" else "sjlt_rows_kernel (S = A R)"
    roofline = {"kernel": kname,
                "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes}

    line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * elapsed / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": w["name"], "n": n, "d": w["d"], "alpha": w["alpha"], "h": w["h"],
                       "adaptive": {k: w[k] for k in ("d0", "dd", "d_max", "eps_rel", "eps_abs")},
                       "passes_over_A_per_step": passes // max(1, args.steps),
                       "l2": "inputs larger than L2 (A = 4.29 GB), no flush",
                       "parallelism": f"replicas x{world}"},
            "per_operator": per_op, "time_share": step_share, "roofline": roofline,
            "gpu_launches": int(launches), "clocks": clk}

    # ---- end to end: A from pinned host memory, results back to the host.  Every step copies
    # its A to the device and its results back; the copies run on a copy stream into the other
    # of two device buffers, so the next step's input and the previous step's results move
    # while the current step computes (ordered by events).
    if not args.no_e2e:
        A_host = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        A_host.copy_(A)
        bufs_e = [A, torch.empty_like(A)]
        steps_e = [Step(b, n, prec_dense, timed_events=False, only=args.only) for b in bufs_e]
        outs = [list(se.bufs.values()) + [se.adS, se.adSt] for se in steps_e]
        hosts = [[torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in oo] for oo in outs]
        comp = torch.cuda.current_stream()
        copy = torch.cuda.Stream()
        in_ready = [torch.cuda.Event(), torch.cuda.Event()]
        computed = [None, None]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        copy.wait_stream(comp)
        with torch.cuda.stream(copy):
            bufs_e[0].copy_(A_host, non_blocking=True)
            in_ready[0].record(copy)
        p2 = 0
        for i in range(args.steps):
            b = i % 2
            if i + 1 < args.steps:  # the next step's A, once the step that last used that buffer is done
                with torch.cuda.stream(copy):
                    if computed[1 - b] is not None:
                        copy.wait_event(computed[1 - b])
                    bufs_e[1 - b].copy_(A_host, non_blocking=True)
                    in_ready[1 - b].record(copy)
            comp.wait_event(in_ready[b])
            p2 += steps_e[b].run(1000 + i)
            computed[b] = torch.cuda.Event()
            computed[b].record(comp)
            with torch.cuda.stream(copy):  # this step's results back to the host
                copy.wait_event(computed[b])
                for o, hh in zip(outs[b], hosts[b]):
                    hh.copy_(o, non_blocking=True)
        comp.wait_stream(copy)
        e1.record(comp)
        torch.cuda.synchronize()
        te = reduce_time_max(e0.elapsed_time(e1) / 1e3, world, "cuda")
        line["e2e"] = {"value": round(job_value(bytes_a, p2, world, te), 1), "unit": "GB/s",
                       "h2d_bytes_per_step": bytes_a,
                       "d2h_bytes_per_step": int(sum(o.numel() * o.element_size() for o in outs[0])),
                       "overlap": "next step's H2D and previous step's D2H on a copy stream, two A buffers"}
        del A_host, hosts, bufs_e, steps_e

    # ---- CPU baseline (oracle) on rank 0, N = 1 only; also checks the GPU results
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.only == "all":
        gpu = {}
        seed = w["seed"] + 7919 * (args.warmup + args.steps - 1)
        for name, kind, alpha, prec in (("sjlt", "sjlt_block", w["alpha"], 0), ("srht", "srht", 1, prec_dense),
                                        ("gauss", "gauss", 1, prec_dense)):
            h = jl.sketch_create(kind, n, w["d"], alpha, seed, w["d"])
            S = torch.empty((n, w["d"]), device="cuda")
            St = torch.empty_like(S)
            jl.sketch_apply(h, A, jl.SK_BOTH, prec, S=S, St=St)
            jl.sketch_destroy(h)
            gpu[name] = (S.double().cpu().numpy(), St.double().cpu().numpy())
        cb, errs = cpu_baseline(X, Y, gpu, args.cpu_rows, seed)
        line["cpu_baseline"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in cb.items()}
        for name in errs:
            line["per_operator"][name]["rel_err_vs_oracle"] = float(f"{errs[name]:.3e}")
    # ---- the precision and differentiation workloads, measured in the same run (rank 0, N = 1)
    if rank == 0 and world == 1 and args.only == "all" and not args.no_extra:
        del step, A
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["precision"] = precision_measure(args)
        torch.cuda.empty_cache()
        line["differentiation"] = differentiation_measure(args)
        torch.cuda.empty_cache()
        line["hss"] = hss_measure(args)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def run_reference(args):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    import numpy as np  # noqa: F401

    from paper_2302_01977_gb300 import inputs
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    X = inputs.points(w["n"], seed=w["seed"])
    Y = inputs.points(w["n"], seed=w["seed"] + 1000)
    for i in range(args.warmup):
        cpu_baseline(X, Y, None, args.ref_rows, w["seed"] + i)
    secs, vals = 0.0, []
    for i in range(args.steps):
        cb, _ = cpu_baseline(X, Y, None, args.ref_rows, w["seed"] + 100 + i)
        secs += cb["seconds"]
        vals.append(cb["value"])
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "n": w["n"], "d": w["d"], "alpha": w["alpha"], "h": w["h"],
                       "sample_rows_per_product": args.ref_rows},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


PRECISION = dict(name="precision_fp32_n65536", n=65536, d=512, h=0.05, seed=20230203 + 2, sample_rows=4096)


def precision_measure(args, sample_rows=None):
    """The Gaussian sketch S = A R of the 65536 x 65536 FP32 kernel matrix
    (h = 0.05, A = 17.2 GB) at d = 512 in each arithmetic: FP32 CUDA cores,
    the bf16 split and scaled FP8 on the tensor cores.  Each result's error is
    measured on sampled rows against an FP64 numpy product of A's FP32 values
    (read back from the device, so the error is the sketch's, not the kernel's
    exp) and the operator's dense R (exported from the handle)."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    w = PRECISION
    n, d = w["n"], w["d"]
    sample_rows = sample_rows or w["sample_rows"]
    torch.cuda.set_device(0)
    X = torch.from_numpy(inputs.points(n, seed=w["seed"])).cuda()
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    jl.kernel_matrix(jl.generator(X, X, w["h"], 0.0), A)
    h = jl.sketch_create("gauss", n, d, 1, w["seed"], d)
    rng = np.random.default_rng(w["seed"])
    rows = np.sort(rng.choice(n, sample_rows, replace=False))
    rows_t = torch.from_numpy(rows).cuda()
    hbm, bf16, _, peak_kind = peaks()
    results = {}
    clocks = Clocks(0)
    clocks.start()
    l0 = jl.sketch_launch_count()
    try:
        for name, prec in (("fp32", jl.SK_PREC_NATIVE), ("bf16x2", jl.SK_PREC_BF16X2), ("fp8", jl.SK_PREC_FP8)):
            S = torch.empty((n, d), dtype=torch.float32, device="cuda")
            for _ in range(args.warmup if name != "fp32" else 1):
                jl.sketch_apply(h, A, jl.SK_S, prec, S=S)
            reps = args.steps if name != "fp32" else 1
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                jl.sketch_apply(h, A, jl.SK_S, prec, S=S)
            e1.record()
            torch.cuda.synchronize()
            jl.sketch_device_status(h)
            ms = e0.elapsed_time(e1) / reps
            results[name] = {"ms": round(ms, 3), "gbs_of_A": round(4.0 * n * n / ms / 1e6, 1),
                             "useful_tflops": round(2.0 * n * n * d / ms / 1e9, 1),
                             "S_rows": S.index_select(0, rows_t).cpu().numpy().astype(np.float64)}
            del S
    finally:
        ck = clocks.stop()
    launches = jl.sketch_launch_count() - l0
    A_rows = A.index_select(0, rows_t).cpu().numpy().astype(np.float64)
    del A
    torch.cuda.empty_cache()
    Rd = jl.sketch_export(h, dense=True)["R"]
    jl.sketch_destroy(h)
    t0 = time.perf_counter()
    ref = A_rows @ Rd
    t_ref = time.perf_counter() - t0
    den = float(np.linalg.norm(ref))
    for r in results.values():
        r["rel_err_vs_fp64"] = float(f"{float(np.linalg.norm(r.pop('S_rows') - ref)) / den:.3e}")
    tol = {"fp32": 1e-5, "bf16x2": 1e-5, "fp8": 2e-2}
    for name, r in results.items():
        r["tolerance"] = tol[name]
        r["within_tolerance"] = r["rel_err_vs_fp64"] <= tol[name]
        r["pct_of_bf16_peak"] = round(100 * r["useful_tflops"] / bf16, 1)
    return {"config": {"workload": w["name"], "n": n, "d": d, "h": w["h"], "operator": "gaussian", "which": "S",
                       "error_sample_rows": int(sample_rows), "l2": "inputs larger than L2 (A = 17.2 GB)"},
            "per_precision": results,
            "bf16x2_speedup_vs_fp32": round(results["fp32"]["ms"] / results["bf16x2"]["ms"], 2),
            "peak_bf16_tflops": bf16, "peak_source": peak_kind,
            "fp64_seconds_on_sample": round(t_ref, 1), "gpu_launches": int(launches), "clocks": ck}


def run_precision(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    m = precision_measure(args)
    best = m["per_precision"]["bf16x2"]
    line = {"metric": METRIC, "value": best["gbs_of_A"], "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 data; bf16 split", "data": "synthetic", "impl": "ours"}
    line.update(m)
    print(json.dumps(line))


DIFF = dict(name="kernel_sketch_grad_n262144", n=262144, d=256, alpha=4, h=0.05, seed=20230203 + 4)


# ALU work per kernel pair (i, j) as the kernels issue it: the forward computes
# K_ij in 7 FP32 operations (3 differences, 2 FMAs and a product for r^2, the
# scale) and one MUFU ex2, and the sketch sum adds alpha = 4 FMAs; the adjoint
# spends 17 FP32 operations on the pair's K_ij, weight and five running sums,
# 4 on G_ij = sum_k s dS[i, c_k], and one ex2.  Peaks are derived from the unit
# counts (128 FP32 lanes and 16 MUFU lanes per SM per clock), the SM count and
# the SM clock sampled during the run.
ALU_OPS = {"forward": (11, 1), "adjoint": (21, 1)}


def differentiation_measure(args, n=None, subset=4096):
    """Matrix-free S = K(X, X; h) R (K never formed) and its adjoint (dX, dh)
    for 262144 points uniform in [0,1]^3, h = 0.05, block SJLT d = 256,
    alpha = 4, upstream dS ~ N(0, 1); against the explicit-K plain path (the
    generator mode of sketch_apply: K written block by block, 20480 rows at a
    time, then the SJLT S = A R product of each block).  On a `subset`-point
    problem of the same kind, the forward and the gradient are also checked
    against the FP64 oracle (oracle.kernel_grad)."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    w = dict(DIFF)
    if n:
        w["n"] = n
        w["name"] = f"kernel_sketch_grad_n{n}"
    n, d = w["n"], w["d"]
    torch.cuda.set_device(0)
    X = torch.from_numpy(inputs.points(n, seed=w["seed"]).astype("float32")).cuda()
    op = jl.Sketch("sjlt_block", n, d, w["alpha"], w["seed"] + 3)
    S = torch.empty((n, d), device="cuda")
    S2 = torch.empty((n, d), device="cuda")
    dS = torch.randn((n, d), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    dX = torch.empty_like(X)
    dh = torch.empty(1, dtype=torch.float64, device="cuda")
    gen = jl.generator(X, X, w["h"])

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    clocks = Clocks(0)
    clocks.start()
    l0 = jl.sketch_launch_count()
    t_fwd = timed(lambda: jl.sketch_kernel_apply(op.h, X, X, w["h"], S), args.steps)
    t_adj = timed(lambda: jl.sketch_kernel_adjoint(op.h, X, w["h"], dS, dX, dh), args.steps)
    launches = jl.sketch_launch_count() - l0
    t_exp = timed(lambda: jl.sketch_apply(op.h, gen, jl.SK_S, 0, S=S2), 1)
    ck = clocks.stop()
    jl.sketch_device_status(op.h)
    fwd_err = float((torch.linalg.norm(S - S2) / torch.linalg.norm(S2)).item())
    op.close()
    del S, S2, dS, dX
    pairs = float(n) * n
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = ck.get("sm_mhz") or 2070.0
    fp32_rate, xu_rate = sms * 128 * mhz * 1e6, sms * 16 * mhz * 1e6
    alu = {}
    for name, t in (("forward", t_fwd), ("adjoint", t_adj)):
        fo, xo = ALU_OPS[name]
        floor_ms = 1e3 * max(fo * pairs / fp32_rate, xo * pairs / xu_rate)
        alu[name] = {"fp32_ops_per_pair": fo, "ex2_per_pair": xo, "floor_ms": round(floor_ms, 2),
                     "frac": round(floor_ms / t, 3)}
    # CPU baseline leg: the FP64 oracle (oracle.kernel_grad) timed on a subset-point problem of the
    # same kind, and the GPU forward and gradient of that problem checked against it
    cb = None
    if not args.no_cpu_baseline:
        from oracle import kernel_grad as okg
        Xs = inputs.points(subset, seed=w["seed"] + 11).astype(np.float32)
        Xt = torch.from_numpy(Xs).cuda()
        ops_ = jl.Sketch("sjlt_block", subset, d, w["alpha"], w["seed"] + 13)
        Ss = torch.empty((subset, d), device="cuda")
        dSs = torch.randn((subset, d), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
        dXs = torch.empty_like(Xt)
        dhs = torch.empty(1, dtype=torch.float64, device="cuda")
        jl.sketch_kernel_apply(ops_.h, Xt, Xt, w["h"], Ss)
        jl.sketch_kernel_adjoint(ops_.h, Xt, w["h"], dSs, dXs, dhs)
        torch.cuda.synchronize()
        R = jl.sketch_export(ops_.h, dense=True)["R"]
        ops_.close()
        X64 = Xs.astype(np.float64)
        dS64 = dSs.double().cpu().numpy()
        t0 = time.perf_counter()
        S0 = okg.kernel_sketch(X64, w["h"], R)
        gX, gh = okg.kernel_sketch_grad(X64, w["h"], R, dS64)
        dt = time.perf_counter() - t0
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        cb = {"value": round(float(subset) * subset / dt / 1e9, 4), "unit": "G kernel pairs/s (forward + adjoint)",
              "cores": cores, "kind": "oracle",
              "sample": f"{subset}-point problem of the same kind (forward S and gradient dX, dh in FP64), {dt:.1f} s",
              "gpu_rel_err": {
                  "forward": float(f"{np.linalg.norm(Ss.double().cpu().numpy() - S0) / np.linalg.norm(S0):.3e}"),
                  "dX": float(f"{np.linalg.norm(dXs.double().cpu().numpy() - gX) / np.linalg.norm(gX):.3e}"),
                  "dh": float(f"{abs(float(dhs.item()) - gh) / abs(gh):.3e}"),
                  "tolerances": {"forward": 1e-5, "gradient": 1e-4}}}
    return {"config": {"workload": w["name"], "n": n, "d": d, "alpha": w["alpha"], "h": w["h"],
                       "upstream": "dS ~ N(0,1)", "l2": "A never formed; X (3 MB) and dS (268 MB)"},
            "forward_ms": round(t_fwd, 3), "adjoint_ms": round(t_adj, 3),
            "explicit_k_forward_ms": round(t_exp, 3), "forward_speedup_vs_explicit": round(t_exp / t_fwd, 2),
            "forward_rel_diff_vs_explicit": float(f"{fwd_err:.3e}"),
            "forward_gpairs_per_s": round(pairs / t_fwd / 1e6, 1),
            "adjoint_gpairs_per_s": round(pairs / t_adj / 1e6, 1),
            "roofline": {"bound": "alu", "unit": "ms", "peak_source": f"derived: {sms} SMs x (128 FP32, 16 MUFU) "
                                                                      f"lanes x {mhz:.0f} MHz sampled", **alu},
            "cpu_baseline": cb, "gpu_launches": int(launches), "clocks": ck}


def run_differentiation(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    m = differentiation_measure(args, n=args.points or None)
    line = {"metric": METRIC, "value": round(m["forward_gpairs_per_s"] * m["adjoint_gpairs_per_s"]
                                             / (m["forward_gpairs_per_s"] + m["adjoint_gpairs_per_s"]), 1),
            "unit": "G kernel pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(m["forward_ms"] + m["adjoint_ms"], 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "ours"}
    line.update(m)
    print(json.dumps(line))


HSS = dict(name="hss_fp64_n2048", n=2048, leaf=64, alpha=4, h=0.2, shift=1e-2, d0=96, dd=32, d_max=512,
           eps_rel=1e-6, eps_abs=0.0, seed=20230203)
HSS_LARGE = dict(HSS, name="hss_fp64_n16384", n=16384, leaf=256, d_max=1024)
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 FP64 (nominal, per GPU)


def hss_measure(args, w=None, cpu=True):
    """Algorithm 1's per-node adaptive loop (hss_compress_adaptive) on a
    symmetric FP64 Gaussian kernel matrix A_ij = exp(-|x_i - x_j|^2 / (2 h^2))
    + shift [i == j] of points uniform in [0,1]^3 ordered by recursive median
    bisection (leaf 64 at n = 2048, the covariance-type problem's shapes; leaf
    256 at n = 16384), block SJLT alpha = 4, d0 = 96, Delta-d = 32,
    eps_rel = 1e-6.  One step = one whole compression (global sketch, every
    sweep, every node), timed with CUDA events around the call; the call's
    own per-kind device times (hss_profile) give the roofline of its dominant
    kernel against the nominal FP64 rate.  The CPU baseline is oracle.hss on
    the same n = 2048 problem."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    w = dict(w or HSS)
    n = w["n"]
    torch.cuda.set_device(0)
    X = inputs.points(n, seed=w["seed"]).astype(np.float64)
    X = X[inputs.bisection_order(X, w["leaf"])]
    Xd = torch.from_numpy(X).cuda()
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    jl.kernel_matrix(jl.generator(Xd, Xd, w["h"], w["shift"]), A)
    torch.cuda.synchronize()

    def once():
        return jl.Hss(A, w["leaf"], "sjlt_block", w["d0"], w["dd"], w["alpha"], w["seed"], w["d_max"],
                      w["eps_rel"], w["eps_abs"])

    for _ in range(args.warmup):
        once().close()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    times, profs = [], []
    l0 = jl.sketch_launch_count()
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        H = once()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        profs.append(H.profile())
        info = H.info()
        ranks = [H.node(i)["k"] for i in range(1, info["nodes"])]
        H.close()
    launches = (jl.sketch_launch_count() - l0) / args.steps
    ck = clocks.stop()
    ms = statistics.median(times)
    kinds = jl.Hss.PROFILE_KINDS
    prof = {k: {"ms": round(statistics.median(p[k]["ms"] for p in profs), 3),
                "gflop": round(profs[0][k]["flops"] / 1e9, 3),
                "launches": profs[0][k]["launches"],
                "avg_sms": round(statistics.median(p[k]["avg_sms"] for p in profs), 1)} for k in kinds}
    for k in kinds:
        prof[k]["gflops"] = round(prof[k]["gflop"] / prof[k]["ms"] * 1e3, 1) if prof[k]["ms"] > 0 else None
    dev_ms = sum(prof[k]["ms"] for k in kinds)
    top = max((k for k in kinds if k != "gather"), key=lambda k: prof[k]["ms"])
    mhz = ck.get("sm_mhz") or 2070.0
    out = {"config": {"workload": w["name"], "n": n, "leaf": w["leaf"], "operator": "sjlt_block",
                      "alpha": w["alpha"], "h": w["h"], "shift": w["shift"], "d0": w["d0"], "dd": w["dd"],
                      "d_max": w["d_max"], "eps_rel": w["eps_rel"], "order": "recursive median bisection",
                      "dtype": "f64"},
           "ms_per_compression": round(ms, 3), "device_ms_by_kind": prof,
           "host_and_gaps_ms": round(ms - dev_ms, 3),
           "d": info["d"], "sweeps": info["sweeps"], "converged": info["converged"], "tests": info["tests"],
           "nodes": info["nodes"], "max_rank": max(ranks) if ranks else 0,
           "gpu_launches": int(launches),
           "roofline": {"kernel": top, "bound": "alu", "unit": "GFLOP/s",
                        "achieved": prof[top]["gflops"], "peak": FP64_NOMINAL_GFLOPS,
                        "frac": round((prof[top]["gflops"] or 0) / FP64_NOMINAL_GFLOPS, 4),
                        "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)", "traffic": None,
                        # the same rate against the FP64 peak of the SMs the kernel's clusters held
                        "avg_sms_held": prof[top]["avg_sms"],
                        "frac_of_held_sms": round((prof[top]["gflops"] or 0) / (FP64_NOMINAL_GFLOPS * max(
                            prof[top]["avg_sms"], 1e-9) / torch.cuda.get_device_properties(0).multi_processor_count),
                            4)},
           "clocks": ck}
    if cpu and not args.no_cpu_baseline:
        from oracle import hss as ohss
        Ah = A.cpu().numpy()
        t0 = time.perf_counter()
        ref = ohss.compress_adaptive(Ah, w["leaf"], "sjlt_block", w["d0"], w["dd"], w["alpha"], w["seed"],
                                     w["d_max"], w["eps_rel"], w["eps_abs"])
        dt = time.perf_counter() - t0
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        out["cpu_baseline"] = {"value": round(dt * 1e3, 1), "unit": "ms per compression", "cores": cores,
                               "kind": "oracle", "sample": f"the whole n = {n} compression (oracle.hss, FP64)",
                               "same_d_and_sweeps": bool(ref["d"] == info["d"] and ref["sweeps"] == info["sweeps"])}
    del A
    torch.cuda.empty_cache()
    return out


def run_hss(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = HSS_LARGE if args.workload == "hss_fp64_n16384" else HSS
    m = hss_measure(args, w, cpu=w is HSS)
    line = {"metric": "per-node adaptive HSS compression time (Algorithm 1)", "value": m["ms_per_compression"],
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": m["ms_per_compression"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "ours"}
    line.update(m)
    print(json.dumps(line))


BATCH = dict(name="batch_kernel_fp32_1024", count=1024, n_lo=256, n_hi=4096, h_lo=0.05, h_hi=0.5,
             d0=(64, 128, 256), dd=32, alpha=4, rounds=3, seed=20230203 + 3)


def run_batching(args):
    """1024 independent FP32 Gaussian kernel matrices A_i = K(X_i, X_i; h_i),
    n_i uniform over multiples of 64 in [256, 4096], h_i uniform in [0.05, 0.5],
    points uniform in [0,1]^3; block SJLT (alpha = 4) with d0_i in {64, 128, 256}
    and Delta-d = 32.  One batched launch sketches Algorithm 1's first d0_i + 32
    columns of every instance; then increments of 32 columns run as replays of a
    captured CUDA graph of the same launch.  value = bytes of all A_i streamed per
    run / run time (A_i is symmetric, so S_i = A_i R_i = A_i^T R_i).  The same
    instances are then sketched with SRHT operators by the batched row transform
    (first sketch and graph-replayed increments, reported under "srht")."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = dict(BATCH)
    if args.instances:
        w["count"] = args.instances
        w["name"] = f"batch_kernel_fp32_{args.instances}"
    torch.cuda.set_device(0)
    rng = np.random.default_rng(w["seed"])
    ns = 64 * rng.integers(w["n_lo"] // 64, w["n_hi"] // 64 + 1, size=w["count"])
    hs = rng.uniform(w["h_lo"], w["h_hi"], size=w["count"])
    d0s = rng.choice(w["d0"], size=w["count"])
    dd, R = w["dd"], w["rounds"]
    ops, As, Sts = [], [], []
    for i in range(w["count"]):
        n = int(ns[i])
        X = torch.from_numpy(inputs.points(n, seed=w["seed"] + 17 * i)).cuda()
        A = torch.empty((n, n), device="cuda")
        jl.kernel_matrix(jl.generator(X, X, float(hs[i])), A)
        # Algorithm 1: the first operator is one JL(d0 + Delta-d), then R increments of Delta-d
        op = jl.Sketch("sjlt_block", n, int(d0s[i]) + dd, w["alpha"], w["seed"] + i,
                       d_max=int(d0s[i]) + (R + 1) * dd)
        for _ in range(R):
            jl.sketch_increment(op.h, dd)
        ops.append(op)
        As.append(A)
        Sts.append(torch.empty((n, int(d0s[i]) + (R + 1) * dd), device="cuda"))
    bytes_a = float(sum(int(n) * int(n) * 4 for n in ns))
    items = [(op.h, A, St, 0, int(d0) + dd) for op, A, St, d0 in zip(ops, As, Sts, d0s)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = jl.Batch(items)
    t_create = time.perf_counter() - t0
    info = B.info()
    clocks = Clocks(0)
    clocks.start()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    l0 = jl.sketch_launch_count()
    t_first = timed(B.run, args.steps)
    launches_first = (jl.sketch_launch_count() - l0) / (args.steps + args.warmup)
    B.status()
    # error of the first sketch on a seeded sample of instances, against an FP64 numpy A^T R
    errs = []
    for i in rng.choice(w["count"], 4, replace=False):
        Rd = jl.sketch_export(ops[i].h, dense=True)["R"]
        hi = int(d0s[i]) + dd
        ref = (As[i].double().cpu().numpy().T @ Rd)[:, :hi]
        got = Sts[i][:, :hi].double().cpu().numpy()
        errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    # increments: a captured graph of the batched launch, replayed with new column ranges
    first_info = info
    B.set(None, [int(d0) + dd for d0 in d0s], [int(d0) + 2 * dd for d0 in d0s])
    B.tune()  # the shape for Delta-d = 32 columns
    info = B.info()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        B.run(stream=s)
    s.synchronize()
    with torch.cuda.graph(g, stream=s):
        B.run(stream=s)
    inc_ms = []
    for r in range(1, R + 1):
        torch.cuda.synchronize()
        B.set(None, [int(d0) + r * dd for d0 in d0s], [int(d0) + (r + 1) * dd for d0 in d0s])
        inc_ms.append(timed(g.replay, args.steps))
    B.status()
    B.close()
    # the same instances with SRHT operators: S_i = A_i R_i by the batched row transform
    # (A_i symmetric, so S_i = A_i^T R_i as above); an SRHT samples at most nu_i columns
    sr_ops, sr_items, sr_d0 = [], [], []
    for i in range(w["count"]):
        n = int(ns[i])
        nu = 1 << (n - 1).bit_length()
        d0 = min(int(d0s[i]), nu - (R + 1) * dd)
        op = jl.Sketch("srht", n, d0 + dd, 1, w["seed"] + i, d_max=d0 + (R + 1) * dd)
        for _ in range(R):
            jl.sketch_increment(op.h, dd)
        sr_ops.append(op)
        sr_d0.append(d0)
        sr_items.append((op.h, As[i], Sts[i], 0, d0 + dd))
    SB = jl.SrhtBatch(sr_items)
    sr_first_info = SB.info()
    sr_first = timed(SB.run, args.steps)
    sr_errs = []
    for i in rng.choice(w["count"], 4, replace=False):
        Rd = jl.sketch_export(sr_ops[i].h, dense=True)["R"]
        hi = sr_d0[i] + dd
        ref = (As[i].double().cpu().numpy() @ Rd)[:, :hi]
        got = Sts[i][:, :hi].double().cpu().numpy()
        sr_errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    SB.set([d0 + dd for d0 in sr_d0], [d0 + 2 * dd for d0 in sr_d0])
    s2 = torch.cuda.Stream()
    g2 = torch.cuda.CUDAGraph()
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g2, stream=s2):
        SB.run(stream=s2)
    sr_inc = []
    for r in range(1, R + 1):
        torch.cuda.synchronize()
        SB.set([d0 + r * dd for d0 in sr_d0], [d0 + (r + 1) * dd for d0 in sr_d0])
        sr_inc.append(timed(g2.replay, args.steps))
    SB.close()
    for op in sr_ops:
        op.close()
    ck = clocks.stop()
    hbm, _, _, peak_kind = peaks()
    t_inc = statistics.median(inc_ms)
    t_sr_inc = statistics.median(sr_inc)
    srht = {"first_sketch_ms": round(sr_first, 3), "first_sketch_gbs": round(bytes_a / sr_first / 1e6, 1),
            "first_sketch_pct_hbm": round(100 * bytes_a / sr_first / 1e6 / hbm, 1),
            "increment_graph_replay_ms": round(t_sr_inc, 3), "increment_gbs": round(bytes_a / t_sr_inc / 1e6, 1),
            "increment_pct_hbm": round(100 * bytes_a / t_sr_inc / 1e6 / hbm, 1), "autotune": sr_first_info,
            "rel_err_vs_fp64_sample": [float(f"{e:.3e}") for e in sr_errs],
            "d0_cap": "d0_i <= nu_i - (increments + 1) * dd"}
    line = {"metric": METRIC, "value": round(bytes_a / t_first / 1e6, 1), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_first, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": w["name"], "instances": w["count"], "n_range": [w["n_lo"], w["n_hi"]],
                       "h_range": [w["h_lo"], w["h_hi"]], "d0": list(w["d0"]), "dd": dd, "alpha": w["alpha"],
                       "bytes_of_A": bytes_a, "l2": "inputs larger than L2 (24 GB of A), no flush"},
            "first_sketch_ms": round(t_first, 3), "first_sketch_pct_hbm": round(100 * bytes_a / t_first / 1e6 / hbm, 1),
            "increment_graph_replay_ms": round(t_inc, 3),
            "increment_gbs": round(bytes_a / t_inc / 1e6, 1),
            "increment_pct_hbm": round(100 * bytes_a / t_inc / 1e6 / hbm, 1),
            "launches_per_run": launches_first, "autotune_first": first_info, "autotune_increment": info,
            "batch_create_s": round(t_create, 2),
            "rel_err_vs_fp64_sample": [float(f"{e:.3e}") for e in errs], "peak_source": peak_kind,
            "gpu_launches": int(launches_first * args.steps), "clocks": ck, "srht": srht}
    for op in ops:
        op.close()
    print(json.dumps(line))


BATCH_ADAPT = dict(name="batch_adaptive_fp32_1024", count=1024, n_lo=256, n_hi=4096, h_lo=0.05, h_hi=0.5,
                   d0=(64, 128, 256), dd=32, alpha=4, eps_rel=1e-6, eps_abs=0.0, seed=20230203 + 3)


def run_batch_adaptive(args):
    """Algorithm 1 for 1024 independent FP32 Gaussian kernel matrices (the batch
    workload's instances) on the device: per round one batched SJLT launch over the
    instances still active, the stopping test of Eq. (3.1) per instance (a CTA cluster
    each), and the table update; Delta-d = 32, eps_rel = 1e-6, increments up to d_max_i = n_i
    (R_i grown up front to d_max_i columns).  The whole loop is one captured
    CUDA graph; value = bytes of A_i streamed (one pass per test taken) / run time."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = dict(BATCH_ADAPT)
    if args.instances:
        w["count"] = args.instances
        w["name"] = f"batch_adaptive_fp32_{args.instances}"
    torch.cuda.set_device(0)
    rng = np.random.default_rng(w["seed"])
    ns = 64 * rng.integers(w["n_lo"] // 64, w["n_hi"] // 64 + 1, size=w["count"])
    hs = rng.uniform(w["h_lo"], w["h_hi"], size=w["count"])
    d0s = rng.choice(w["d0"], size=w["count"])
    dd = w["dd"]
    # increments per instance: up to d_max_i = n_i (the configuration as written), or a fixed count
    incs_i = [max(0, (int(ns[i]) - int(d0s[i])) // dd - 1) if not args.max_increments else args.max_increments
              for i in range(w["count"])]  # d_max_i = n_i, and at least d0_i + dd (one test)
    ops, As, Sts = [], [], []
    for i in range(w["count"]):
        n = int(ns[i])
        X = torch.from_numpy(inputs.points(n, seed=w["seed"] + 17 * i)).cuda()
        A = torch.empty((n, n), device="cuda")
        jl.kernel_matrix(jl.generator(X, X, float(hs[i])), A)
        d_max = int(d0s[i]) + (incs_i[i] + 1) * dd
        op = jl.Sketch("sjlt_block", n, int(d0s[i]) + dd, w["alpha"], w["seed"] + i, d_max=d_max)
        for _ in range(incs_i[i]):
            jl.sketch_increment(op.h, dd)
        ops.append(op)
        As.append(A)
        Sts.append(torch.empty((n, d_max), device="cuda"))
    items = [(op.h, A, St, 0, int(d0) + dd) for op, A, St, d0 in zip(ops, As, Sts, d0s)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = jl.Batch(items)
    B.adaptive_setup([int(d) for d in d0s], dd, w["eps_rel"], w["eps_abs"])
    t_setup = time.perf_counter() - t0
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        B.adaptive_run(stream=s)
    s.synchronize()
    l0 = jl.sketch_launch_count()
    with torch.cuda.graph(g, stream=s):
        B.adaptive_run(stream=s)
    launches = jl.sketch_launch_count() - l0
    clocks = Clocks(0)
    clocks.start()
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            g.replay()
    e1.record(s)
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_run = e0.elapsed_time(e1) / args.steps
    res = B.adaptive_result()
    bytes_streamed = float(sum(int(t) * int(n) * int(n) * 4 for t, n in zip(res["tests"], ns)))
    hbm, _, _, peak_kind = peaks()
    # error of the final sketch on a seeded sample of small instances against an FP64 numpy
    # A_i^T R_i[:, :d_i]; R_i exported at d_total carries 1/sqrt(alpha B_total), R_i[:, :d_i] 1/sqrt(alpha B_d)
    errs = []
    small = [i for i in range(w["count"]) if ns[i] <= 1024]
    for i in rng.choice(small, min(3, len(small)), replace=False):
        d = int(res["d"][i])
        blocks_d = 1 + (d - int(d0s[i]) - dd) // dd
        Rd = jl.sketch_export(ops[i].h, dense=True)["R"][:, :d] * np.sqrt((incs_i[i] + 1) / blocks_d)
        ref = As[i].double().cpu().numpy().T @ Rd
        got = Sts[i][:, :d].double().cpu().numpy()
        errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    rounds = int(res["tests"].max())
    line = {"metric": METRIC, "value": round(bytes_streamed / t_run / 1e6, 1), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_run, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": w["name"], "instances": w["count"], "n_range": [w["n_lo"], w["n_hi"]],
                       "h_range": [w["h_lo"], w["h_hi"]], "d0": list(w["d0"]), "dd": dd, "alpha": w["alpha"],
                       "d_max": ("max(n_i, d0_i + dd)" if not args.max_increments
                                 else f"d0_i + {args.max_increments + 1} * dd"),
                       "eps_rel": w["eps_rel"], "eps_abs": w["eps_abs"],
                       "l2": "inputs larger than L2 (24 GB of A), no flush"},
            "adaptive_run_ms": round(t_run, 3), "rounds": rounds,
            "pct_hbm_of_streamed_bytes": round(100 * bytes_streamed / t_run / 1e6 / hbm, 1),
            "bytes_streamed": bytes_streamed,
            "converged": int((res["state"] == 1).sum()), "out_of_increments": int((res["state"] == 2).sum()),
            "still_running": int((res["state"] == 0).sum()),
            "mean_d": round(float(res["d"].mean()), 1), "tests_taken": int(res["tests"].sum()),
            "graph_launches_per_run": int(launches), "setup_s": round(t_setup, 2),
            "autotune": B.info(),
            "rel_err_vs_fp64_sample": [float(f"{e:.3e}") for e in errs], "peak_source": peak_kind,
            "gpu_launches": int(launches * args.steps), "clocks": ck}
    B.close()
    for op in ops:
        op.close()
    line["srht"] = batch_adaptive_srht(args, w, ns, d0s, As, Sts, incs_i)
    print(json.dumps(line))


def batch_adaptive_srht(args, w, ns, d0s, As, Sts, incs_i):
    """The same loop with SRHT operators (S_i = A_i R_i = A_i^T R_i, A_i symmetric): an SRHT
    samples at most nu_i columns, so d0_i <= nu_i - 64 and the increments stop at nu_i (and at
    the SJLT loop's d_max_i)."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import jlsketch as jl

    dd = w["dd"]
    ops, items, d0c = [], [], []
    for i in range(w["count"]):
        n = int(ns[i])
        nu = 1 << (n - 1).bit_length()
        d0 = min(int(d0s[i]), nu - 2 * dd)
        k = min(incs_i[i], (nu - d0) // dd - 1, (Sts[i].shape[1] - d0) // dd - 1)
        op = jl.Sketch("srht", n, d0 + dd, 1, w["seed"] + i, d_max=d0 + (k + 1) * dd)
        for _ in range(k):
            jl.sketch_increment(op.h, dd)
        ops.append(op)
        d0c.append(d0)
        items.append((op.h, As[i], Sts[i], 0, d0 + dd))
    B = jl.SrhtBatch(items)
    B.adaptive_setup(d0c, dd, w["eps_rel"], w["eps_abs"])
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        B.adaptive_run(stream=s)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            g.replay()
    e1.record(s)
    torch.cuda.synchronize()
    t_run = e0.elapsed_time(e1) / args.steps
    res = B.adaptive_result()
    bytes_streamed = float(sum(int(t) * int(n) * int(n) * 4 for t, n in zip(res["tests"], ns)))
    hbm, _, _, _ = peaks()
    out = {"adaptive_run_ms": round(t_run, 3), "gbs_of_streamed_bytes": round(bytes_streamed / t_run / 1e6, 1),
           "pct_hbm_of_streamed_bytes": round(100 * bytes_streamed / t_run / 1e6 / hbm, 1),
           "converged": int((res["state"] == 1).sum()), "out_of_columns": int((res["state"] == 2).sum()),
           "still_running": int((res["state"] == 0).sum()), "tests_taken": int(res["tests"].sum()),
           "mean_d": round(float(res["d"].mean()), 1), "ctas_per_sm": B.info()["ctas_per_sm"],
           "d_cap": "d0_i <= nu_i - 64, d_max_i <= min(nu_i, the SJLT loop's d_max_i)"}
    B.close()
    for op in ops:
        op.close()
    return out


SRHT_SPLIT = dict(name="srht_nonpow2_fp32_n24000", n=24000, d=256, h=0.1, sample_rows=256, seed=20230203 + 6)


def run_srht_split(args):
    """SRHT S = A D H P/sqrt(d) for a non-power-of-two order (n = 24000 = k + r,
    k = 16384, r = 7616, p = 8192) through the row FWHT: Sec. 7.1's split into
    transforms of orders k and p against the transform of rows zero-padded to
    nu = 32768.  A = K(X, Y; h) in FP32 (X != Y, 2.3 GB); value = GB/s of A of
    the split.  Errors on sampled rows against an FP64 numpy A R with the
    exported operator."""
    import numpy as np
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = SRHT_SPLIT
    n, d = w["n"], w["d"]
    torch.cuda.set_device(0)
    X = torch.from_numpy(inputs.points(n, seed=w["seed"])).cuda()
    Y = torch.from_numpy(inputs.points(n, seed=w["seed"] + 1)).cuda()
    ld = (n + 3) // 4 * 4
    Abuf = torch.empty((n, ld), dtype=torch.float32, device="cuda")
    A = Abuf[:, :n]
    jl.kernel_matrix(jl.generator(X, Y, w["h"]), A)
    h = jl.sketch_create("srht", n, d, 1, w["seed"], d)
    rng = np.random.default_rng(w["seed"])
    rows = np.sort(rng.choice(n, w["sample_rows"], replace=False))
    rows_t = torch.from_numpy(rows).cuda()
    hbm, _, _, peak_kind = peaks()
    os.environ["JLS_SRHT_ROUTE"] = "fwht"
    res = {}
    clocks = Clocks(0)
    clocks.start()
    try:
        for name, split in (("split", "1"), ("padded", "0")):
            os.environ["JLS_SRHT_SPLIT"] = split
            S = torch.empty((n, d), dtype=torch.float32, device="cuda")
            for _ in range(args.warmup):
                jl.sketch_apply(h, A, jl.SK_S, S=S)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = jl.sketch_launch_count()
            e0.record()
            for _ in range(args.steps):
                jl.sketch_apply(h, A, jl.SK_S, S=S)
            e1.record()
            torch.cuda.synchronize()
            jl.sketch_device_status(h)
            ms = e0.elapsed_time(e1) / args.steps
            res[name] = {"ms": round(ms, 3), "gbs_of_A": round(4.0 * n * n / ms / 1e6, 1),
                         "pct_hbm": round(100 * 4.0 * n * n / ms / 1e6 / hbm, 1),
                         "launches_per_apply": (jl.sketch_launch_count() - l0) / args.steps,
                         "S_rows": S.index_select(0, rows_t).double().cpu().numpy()}
    finally:
        ck = clocks.stop()
        os.environ.pop("JLS_SRHT_ROUTE", None)
        os.environ.pop("JLS_SRHT_SPLIT", None)
    R = jl.sketch_export(h, dense=True)["R"]
    jl.sketch_destroy(h)
    ref = A.index_select(0, rows_t).double().cpu().numpy() @ R
    for r in res.values():
        r["rel_err_vs_fp64"] = float(f"{np.linalg.norm(r.pop('S_rows') - ref) / np.linalg.norm(ref):.3e}")
    best = res["split"]
    line = {"metric": METRIC, "value": best["gbs_of_A"], "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": w["name"], "n": n, "d": d, "h": w["h"], "operator": "srht", "which": "S",
                       "k": 16384, "r": n - 16384, "p": 8192, "nu": 32768,
                       "l2": "inputs larger than L2 (2.3 GB of A), no flush"},
            "split": res["split"], "padded": res["padded"],
            "speedup_split_vs_padded": round(res["padded"]["ms"] / res["split"]["ms"], 3),
            "peak_source": peak_kind, "gpu_launches": int(res["split"]["launches_per_apply"] * args.steps),
            "clocks": ck}
    print(json.dumps(line))


COMPLEX = dict(name="complex_helmholtz_fp32_n16384", n=16384, d=256, alpha=4, kappa=20.0, seed=20230203 + 5)


def run_complex(args):
    """S = A R and S' = A* R for a complex Helmholtz-type kernel A_ij =
    exp(i kappa r_ij) / (1 + kappa r_ij) of 16384 points uniform in [0,1]^3
    (complex64, 2.1 GB), block SJLT d = 256, alpha = 4 (and SRHT and Gaussian
    operators, d = 256, in the bf16 split).  value = bytes of A / time of the
    SJLT S'."""
    import torch

    from paper_2302_01977_gb300 import inputs
    from paper_2302_01977_gb300 import jlsketch as jl

    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = COMPLEX
    n, d = w["n"], w["d"]
    torch.cuda.set_device(0)
    X = torch.from_numpy(inputs.points(n, seed=w["seed"])).cuda().double()
    A = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    for r0 in range(0, n, 2048):  # input generation in row blocks (torch), not timed
        r = torch.cdist(X[r0:r0 + 2048], X)
        A[r0:r0 + 2048] = (torch.exp(1j * w["kappa"] * r) / (1.0 + w["kappa"] * r)).to(torch.complex64)
    del X
    op = jl.Sketch("sjlt_block", n, d, w["alpha"], w["seed"])
    S = torch.empty((n, d), dtype=torch.complex64, device="cuda")
    St = torch.empty_like(S)
    bytes_a = float(n) * n * 8
    hbm, _, _, peak_kind = peaks()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    clocks = Clocks(0)
    clocks.start()
    l0 = jl.sketch_launch_count()
    t_s = timed(lambda: jl.sketch_apply(op.h, A, jl.SK_S, S=S))
    t_st = timed(lambda: jl.sketch_apply(op.h, A, jl.SK_ST, St=St))
    jl.sketch_device_status(op.h)
    sym = float((torch.linalg.norm(St - S.conj()) / torch.linalg.norm(S)).item())  # A symmetric: A* R = conj(A R)
    op.close()
    # SRHT and Gaussian operators on the same A: the bf16 split on tensor cores (S through R (x) I_2,
    # S' through the transpose product and a conjugating interleave)
    dense = {}
    for kind in ("srht", "gauss"):
        with jl.Sketch(kind, n, d, 1, w["seed"] + 1) as dop:
            ts = timed(lambda: jl.sketch_apply(dop.h, A, jl.SK_S, jl.SK_PREC_BF16X2, S=S))
            tst = timed(lambda: jl.sketch_apply(dop.h, A, jl.SK_ST, jl.SK_PREC_BF16X2, St=St))
            jl.sketch_device_status(dop.h)
        dsym = float((torch.linalg.norm(St - S.conj()) / torch.linalg.norm(S)).item())
        dense[kind] = {"prec": "bf16x2", "S_ms": round(ts, 4), "St_ms": round(tst, 4),
                       "S_gbs": round(bytes_a / ts / 1e6, 1), "St_gbs": round(bytes_a / tst / 1e6, 1),
                       "symmetry_rel_diff": float(f"{dsym:.3e}")}
    launches = jl.sketch_launch_count() - l0
    ck = clocks.stop()
    line = {"metric": METRIC, "value": round(bytes_a / t_st / 1e6, 1), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_s + t_st, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32 parts)",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": w["name"], "n": n, "d": d, "alpha": w["alpha"], "kappa": w["kappa"],
                       "l2": "inputs larger than L2 (A = 2.1 GB), no flush"},
            "S_ms": round(t_s, 4), "St_ms": round(t_st, 4),
            "S_gbs": round(bytes_a / t_s / 1e6, 1), "St_gbs": round(bytes_a / t_st / 1e6, 1),
            "pct_hbm_S": round(100 * bytes_a / t_s / 1e6 / hbm, 1),
            "pct_hbm_St": round(100 * bytes_a / t_st / 1e6 / hbm, 1), "peak_source": peak_kind,
            "symmetry_rel_diff": float(f"{sym:.3e}"), "srht": dense["srht"], "gauss": dense["gauss"],
            "gpu_launches": int(launches), "clocks": ck}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["auto", "fp32", "bf16x2"], default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the precision (n = 65536), differentiation (n = 262144) and per-node HSS (n = 2048) "
                         "sections of the default run")
    ap.add_argument("--cpu-rows", type=int, default=512)
    ap.add_argument("--ref-rows", type=int, default=128)
    ap.add_argument("--n", type=int, default=WORKLOAD["n"],
                    help="matrix order (the benchmark workload is 32768; smaller n for profiling captures)")
    ap.add_argument("--workload", choices=["kernel_fp32_n32768", "precision_fp32_n65536",
                                           "kernel_sketch_grad_n262144", "batch_kernel_fp32_1024",
                                           "batch_adaptive_fp32_1024", "complex_helmholtz_fp32_n16384",
                                           "srht_nonpow2_fp32_n24000", "hss_fp64_n2048", "hss_fp64_n16384"],
                    default="kernel_fp32_n32768",
                    help="the benchmark (default), or the Gaussian precision comparison at n = 65536, d = 512")
    ap.add_argument("--points", type=int, default=0,
                    help="kernel_sketch_grad workload: number of points (default 262144; smaller for captures)")
    ap.add_argument("--max-increments", type=int, default=0,
                    help="batch_adaptive workload: increments per instance (default 0: up to d_max_i = n_i)")
    ap.add_argument("--instances", type=int, default=0,
                    help="batch workload: number of instances (default 1024; fewer for captures)")
    ap.add_argument("--only", choices=["all", "sjlt", "srht", "gauss", "adaptive"], default="all",
                    help="restrict the step (profiling captures); the benchmark runs all")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "precision_fp32_n65536":
        run_precision(args)
    elif args.workload == "kernel_sketch_grad_n262144":
        run_differentiation(args)
    elif args.workload == "batch_kernel_fp32_1024":
        run_batching(args)
    elif args.workload == "batch_adaptive_fp32_1024":
        run_batch_adaptive(args)
    elif args.workload == "srht_nonpow2_fp32_n24000":
        run_srht_split(args)
    elif args.workload == "complex_helmholtz_fp32_n16384":
        run_complex(args)
    elif args.workload in ("hss_fp64_n2048", "hss_fp64_n16384"):
        run_hss(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

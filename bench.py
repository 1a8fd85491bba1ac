#!/usr/bin/env python3
"""Benchmark of the metric-magnitude hot path on GB300.

Workload (default): n = 100,000 points uniform in [0, 1]^8 (seeded), solved at
t in {1, 10, log(n-1)/min d}; one step = those three solves of Zw = 1 to
relative residual <= 1e-14 (generation, factor, triangular solves, FP64
refinement, magnitude).  Metric unit: TFLOP/s of useful work
(n^3/3 + 2 n^2 per refinement step, per solve) over device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica (independent seeded
problem) on its own GPU: weak scaling, no collective on the data path; the
barrier and the max over ranks bracket the timed region.  `--impl reference`
times the CPU FP64 oracle on the host cores on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n=1e5 Zw=1 solve s & TFLOP/s, mixed+IR vs FP64 dense at 1e-14 resid; batch solve/s"
UNIT = "TFLOP/s"


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=100_000)
    p.add_argument("--m", type=int, default=8)
    p.add_argument("--ts", default="1,10,bound", help="comma list of t values; 'bound' = log(n-1)/min d")
    p.add_argument("--precision", default="auto")
    p.add_argument("--resid", default="auto", choices=["auto", "matrix_free", "stored"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--extras", action="store_true", help="also time sweep/grad/batch/FP64 comparators")
    p.add_argument("--cpu-sample-n", type=int, default=12288)
    p.add_argument("--panel-tiles", type=int, default=0, help="factor panel width in 128-wide tiles (0 = library default)")
    p.add_argument("--lookahead", type=int, default=1, help="1: factor the next panel on a second stream")
    p.add_argument("--lookahead-sms", type=int, default=0, help="> 0: SMs kept for the panel stream; 0: library default (stream priority); < 0: priority with that many trailing blocks per CTA")
    p.add_argument("--paper-sweep", action="store_true",
                   help="instead of the headline step: the paper's runtime workload (t_+ and w(t_+) for "
                        "n in 1e3..3e4, m in 3..100, two covariances, 3 runs) with bisection and Ridders")
    p.add_argument("--batch-only", action="store_true",
                   help="instead of the headline step: time the batched solver (512 clouds in R^32 x 8 t)")
    p.add_argument("--no-comparators", action="store_true",
                   help="skip the FP64-dense comparison and the batch throughput after the timed steps")
    p.add_argument("--fp64-dense-n", type=int, default=0,
                   help="instead of the headline step: the FP64 dense paths against AUTO at this n "
                        "(points uniform in [0,1]^8, t=1; --no-cusolver to skip cuSOLVER)")
    p.add_argument("--no-cusolver", action="store_true")
    p.add_argument("--ooc-n", type=int, default=0,
                   help="instead of the headline step: one solve of n points in [0,1]^8 at --ts' first t with the "
                        "default options (out of core when the FP32 tiles do not fit in device memory)")
    p.add_argument("--cta-pairs", type=int, default=1,
                   help="CTA-pair (cta_group::2) tensor-core updates: 1 always, 0 never, 2 split precisions only")
    return p.parse_args()


# ----------------------------------------------------------------- helpers
def dist_env():
    from paper_2607_23354_gb300 import replicas
    return replicas.rank_world()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """The committed ncu DRAM-traffic record of the dominant kernel, or None
    when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not d:
        return None
    try:
        if source_hash(d["sources"]) != d["source_hash"]:
            return None
    except (OSError, KeyError):
        return None
    return d


def cpu_oracle_sample(X, t, n_s):
    """Time the CPU oracle (as it stands) on a seeded n_s-point subset: one
    weighting solve (Z, Cholesky, 2 refinement steps)."""
    import oracle
    import workloads
    Xs = workloads.subsample(X, n_s, seed=11)
    t0 = time.perf_counter()
    w, mag, info = oracle.weighting(Xs, t, ir_steps=2)
    el = time.perf_counter() - t0
    flops = n_s ** 3 / 3 + 2 * n_s ** 2 * 2
    return {"value": flops / el / 1e12, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n_s} of the {X.shape[0]} points (seeded subset), m={X.shape[1]}, t={t:g}: one oracle "
                      f"solve (Z, Cholesky, forward/back substitution, 2 FP64 refinement steps) in {el:.2f} s",
            "seconds": el, "rel_residual": info["rel_residual"]}


# --------------------------------------------------------------- our arm
def run_ours(a):
    import numpy as np
    import torch

    import paper_2607_23354_gb300 as M
    import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    X = workloads.unit_cube_cloud(n=a.n, m=a.m, seed=workloads.SEEDS["cube"] + rank)
    Xd = torch.from_numpy(X).to(dev)
    opts = M.Options(precision=a.precision, residual_mode=a.resid, profile=True, panel_tiles=a.panel_tiles,
                     lookahead=bool(a.lookahead), lookahead_sms=a.lookahead_sms, cta_pairs=a.cta_pairs)
    ctx = M.Context(opts)
    # 'bound' = the Sec. 1 bound log(n-1)/min d, found inside the call (t <= 0
    # asks mag_solve_multi for it: min d comes from the first t's generator)
    ts = [0.0 if s.strip() == "bound" else float(s) for s in a.ts.split(",")]
    Wbuf = torch.empty(len(ts), a.n, dtype=torch.float64, device=dev)

    def step(acc=None):
        # one call for the step's t values: distances are computed once per
        # call (and freed with it), Z and the factor once per t
        _, mags, infos_t = ctx.solve_multi(Xd, ts, W=Wbuf)
        if acc is not None:
            acc.extend(zip(ts, mags, infos_t))

    for _ in range(a.warmup):
        step()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id)
    stream = torch.cuda.current_stream(dev)
    infos = []
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step(infos)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    from paper_2607_23354_gb300 import replicas
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), device=dev)
    flops_step = sum(i["useful_flops"] for _, _, i in infos) / a.steps
    value = world * flops_step * a.steps / (ms / 1e3) / 1e12

    # e2e: host (pinned) points in, host w out, copies inside the timed region
    e2e = None
    if not a.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        Xe = torch.empty_like(Xd)
        h2d = Xh.numel() * 8
        d2h = a.n * 8 * len(ts)
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f2 = 0.0
        Wh = torch.empty(len(ts), a.n, dtype=torch.float64).pin_memory()
        for _ in range(a.steps):
            Xe.copy_(Xh, non_blocking=True)
            _, mags, infos_t = ctx.solve_multi(Xe, ts, W=Wbuf)
            Wh.copy_(Wbuf, non_blocking=True)
            f2 += sum(i["useful_flops"] for i in infos_t)
            torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        barrier()
        el = replicas.max_over_ranks(el, device=dev)
        e2e = {"value": world * f2 / el / 1e12, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h + 8 * len(ts)}

    out = None
    if rank == 0:
        peaks, peak_kind = measured_peaks()
        last = infos[-len(ts):]
        dmin = last[0][2]["min_distance"]
        per_t = [{"t": i["t"], "solve_s": i["ms_total"] / 1e3, "mag": mag, "rel_residual": i["rel_residual"],
                  "ir_iters": i["ir_iters"], "gmres_iters": i["gmres_iters"], "precision_used": i["precision_used"],
                  "fallback": i["fallback"],
                  "ms_generate": i["ms_generate"], "ms_factor": i["ms_factor"], "ms_solve": i["ms_solve"],
                  "ms_residual": i["ms_residual"], "residual_evals": i["residual_evals"],
                  "residual_evals_ff": i["residual_evals_ff"],
                  "probe_rho": i["probe_rho"], "ms_probe": i["ms_probe"],
                  "ms_factor_parts": {"update_trailing": i["ms_update"] - i["ms_update_panel"],
                                      "update_panel": i["ms_update_panel"], "potrf": i["ms_potrf"],
                                      "trsm": i["ms_trsm"], "split": i["ms_split"],
                                      "update_busy": i["ms_update_busy"]}} for t, mag, i in last]
        upd_ms = sum(i["ms_update"] for _, _, i in infos)
        # wall time with at least one update launch in flight: the look-ahead
        # factor's two streams run update launches at the same time, and the
        # sum of their intervals counts those stretches twice
        busy_ms = sum(i["ms_update_busy"] for _, _, i in infos)
        upd_launch = sum(i["update_launches"] for _, _, i in infos)
        upd_flops = sum(i["update_flops"] for _, _, i in infos)
        prec_used = {i["precision_used"] for _, _, i in infos}
        tensor = any(p in (M.PREC_BF16, M.PREC_TF32, M.PREC_TF32X3, M.PREC_FP16X3, M.PREC_FP16)
                     for p in prec_used)
        f16 = all(p in (M.PREC_BF16, M.PREC_FP16X3, M.PREC_FP16) for p in prec_used)
        smx = peaks.get("sm_max_mhz", 2070.0)
        # the update kernel runs inside a seconds-long step: sustained tensor peak
        bf16, bf16_kind = peaks.get("bf16_tflops_sustained"), "sustained"
        if not bf16:
            bf16, bf16_kind = peaks["bf16_tflops"], "burst"
        if tensor and f16:
            peak = bf16  # FP16 and BF16 dense tensor rates are equal (nominal 2.25 PF each)
            bound, kname = "tensor", "trailing_update_tc"
            peak_note = (f"FP16 tensor peak = {peak_kind} {bf16_kind} BF16 {bf16} TF/s "
                         f"(equal nominal FP16/BF16 rates)")
        elif tensor:
            peak = bf16 * (1.1 / 2.25)  # TF32 dense / BF16 dense, nominal ratio
            bound, kname = "tensor", "trailing_update_tc"
            peak_note = (f"TF32 tensor peak = {peak_kind} {bf16_kind} BF16 {bf16} TF/s x nominal "
                         f"TF32/BF16 ratio 1.1/2.25")
        else:
            peak = 152 * 128 * 2 * smx * 1e6 / 1e12
            bound, kname = "alu", "trailing_update_simt"
            peak_note = f"FP32 FMA peak = 152 SMs x 128 lanes x 2 flops x {smx:.0f} MHz"
        achieved = (upd_flops / upd_launch) / ((busy_ms / upd_launch) / 1e3) / 1e12 if upd_launch and busy_ms else None
        achieved_sum = (upd_flops / upd_launch) / ((upd_ms / upd_launch) / 1e3) / 1e12 if upd_launch else None
        # split precisions execute three tensor products per useful product
        split = (M.PREC_FP16X3, M.PREC_TF32X3)
        exec_flops = sum(i["update_flops"] * (3 if i["precision_used"] in split else 1) for _, _, i in infos)
        executed = exec_flops / (busy_ms / 1e3) / 1e12 if busy_ms else None
        # bytes per algorithmic flop of each precision's launches (ncu records of
        # smaller captures) x this run's flops of that precision, per launch
        trec = {M.PREC_FP16X3: ncu_traffic(kname), M.PREC_FP16: ncu_traffic(kname + "_fp16")}
        traffic = None
        if upd_launch and all(trec.get(i["precision_used"]) for _, _, i in infos if i["update_flops"]):
            traffic = sum(trec[i["precision_used"]]["bytes_per_flop"] * i["update_flops"]
                          for _, _, i in infos if i["update_flops"]) / upd_launch
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                    "kernel": kname, "launches": upd_launch, "avg_launch_ms": busy_ms / max(upd_launch, 1),
                    "flops_per_launch": upd_flops / max(upd_launch, 1), "peak_source": peak_note,
                    "executed_tflops": executed,
                    "executed_frac": (executed / peak) if executed else None,
                    "sum_of_intervals": {"avg_launch_ms": upd_ms / max(upd_launch, 1), "achieved": achieved_sum,
                                         "frac": (achieved_sum / peak) if achieved_sum else None},
                    "note": "achieved = algorithmic flops (2*128^3 per tile product) of every update launch of the "
                            "timed steps / the wall time during which at least one of them was in flight (the "
                            "union of their CUDA-event intervals on both streams of the look-ahead factor; "
                            "avg_launch_ms = that time / launches); sum_of_intervals divides by the plain sum "
                            "of the intervals instead, which counts the overlap of the two streams twice; "
                            "executed counts the 3 tensor products per useful one of FP16X3/TF32X3",
                    "share_of_step": busy_ms / ms if ms else None}
        launches = sum(i["kernel_launches"] for _, _, i in infos)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": f"n={a.n} points uniform in [0,1]^{a.m} (seed {workloads.SEEDS['cube']}+rank), "
                                      f"t in {{{', '.join(s.strip() for s in a.ts.split(','))}}}; one step = "
                                      f"{len(ts)} solves to rel. residual <= 1e-14 (the bound log(n-1)/min d "
                                      f"found inside the step)",
                          "n": a.n, "m": a.m, "t": [i["t"] for _, _, i in last], "precision": a.precision,
                          "residual_mode": a.resid,
                          "panel_tiles": a.panel_tiles or "auto (16 split, 32 one-product)",
                          "parallelism": f"replicas x{world}",
                          "l2": "inputs larger than L2 (packed factor tiles of several GB per solve)",
                          "api": "mag_solve_multi (one call per step for all t; distances computed once per call)"},
               "solve_s": sum(p["solve_s"] for p in per_t), "per_t": per_t,
               "roofline": roofline, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
               "min_distance": dmin}
    return out, (ctx, Xd, X, ts)


def _gpu_id(dev):
    import torch
    props = torch.cuda.get_device_properties(dev)
    gid = str(getattr(props, "uuid", dev.index))
    if gid and not gid.startswith("GPU-") and len(gid) > 8:
        gid = "GPU-" + gid
    return gid


def _event_time(fn, dev):
    """Device time (s) of fn() on the current stream, host-synchronised on both sides."""
    import torch
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / 1e3, r


def fp64_dense_comparison(dev, n=16384, t=0.5, repeats=3):
    """The metric's comparison: mixed precision + FP64 refinement (AUTO) against
    the plain FP64 dense path on the same GPU -- this library's FP64 blocked
    Cholesky (precision = fp64, CUDA-core FP64) and cuSOLVER's FP64 Cholesky
    (torch.linalg.cholesky + cholesky_solve on the full square matrix) -- on
    the precision workload (Gaussian mixture, n = 16384 in R^3, t = 0.5).
    Device-timed, `repeats` runs each after one warm-up, clocks sampled."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    X = torch.from_numpy(workloads.gaussian_mixture_cloud(n=n)).to(dev)
    sampler = ClockSampler(_gpu_id(dev))
    res = {"workload": f"Gaussian mixture n={n} in R^3 (seed {workloads.SEEDS['mixture']}), t={t}",
           "n": n, "t": t, "repeats": repeats}
    sampler.start()
    for prec in ("auto", "fp64"):
        c = M.Context(M.Options(precision=prec))
        c.solve(X, t)
        times, info = [], None
        for _ in range(repeats):
            el, (_, _, info) = _event_time(lambda: c.solve(X, t), dev)
            times.append(el)
        res[f"{prec}_s"] = times
        res[f"{prec}_rel_residual"] = info["rel_residual"]
        res[f"{prec}_ir_iters"] = info["ir_iters"]
        c.close()
    try:
        def cusolver():
            d = torch.cdist(X, X)
            Z = torch.exp(d.mul_(-t))
            del d
            L = torch.linalg.cholesky(Z)
            w = torch.cholesky_solve(torch.ones(n, 1, dtype=torch.float64, device=dev), L)
            return w
        cusolver()
        times = []
        for _ in range(repeats):
            el, w = _event_time(cusolver, dev)
            times.append(el)
        res["cusolver_fp64_s"] = times
        del w
        torch.cuda.empty_cache()
    except Exception as e:  # noqa: BLE001
        res["cusolver_fp64_error"] = str(e)[:160]
    res["clocks"] = sampler.stop()
    best = {k: min(v) for k, v in res.items() if k.endswith("_s") and isinstance(v, list)}
    res["best_s"] = best
    res["speedup_vs_own_fp64"] = best["fp64_s"] / best["auto_s"]
    if "cusolver_fp64_s" in best:
        res["speedup_vs_cusolver_fp64"] = best["cusolver_fp64_s"] / best["auto_s"]
    return res


def batch_throughput(dev, repeats=3):
    """Batch solves/s: 512 clouds in R^32 (sizes log-uniform in [64, 2048]) x 8
    values of t in [0.1, 10], one persistent solve launch per call
    (mag_solve_batch), device-timed after one warm-up; best of `repeats`."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    c = M.Context(M.Options())
    clouds, tvals = workloads.batch_clouds()
    cl = [torch.from_numpy(x).to(dev) for x in clouds]
    c.solve_batch(cl, list(tvals))
    times, failed = [], 0
    for _ in range(repeats):
        el, (_, _, sts) = _event_time(lambda: c.solve_batch(cl, list(tvals)), dev)
        times.append(el)
        failed = int((sts != 0).sum())
    c.close()
    nsolves = len(cl) * len(tvals)
    return {"workload": "512 clouds in R^32, n log-uniform in [64, 2048], x 8 t log-spaced in [0.1, 10]",
            "solves": nsolves, "seconds": times, "solves_per_s": nsolves / min(times), "failed": failed}


def run_extras(ctx, a, out, Xd):
    """Bounded side measurements: FP64 dense comparators, sweep, gradients, batch."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    ex = {}
    # FP64 dense on the same GPU at the precision config's size (n = 16384)
    Xm = torch.from_numpy(workloads.gaussian_mixture_cloud()).cuda()
    for prec in ["fp64", "auto"]:
        ctx.set_options(M.Options(precision=prec))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, mag, info = ctx.solve(Xm, 0.5)
        torch.cuda.synchronize()
        ex[f"mixture_n16384_t0.5_{prec}_s"] = time.perf_counter() - t0
    ctx.set_options(M.Options(precision=a.precision, residual_mode=a.resid, profile=True))
    try:
        Zc = None
        n2 = Xm.shape[0]
        d = torch.cdist(Xm, Xm)
        Zc = torch.exp(-0.5 * d)
        del d
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = torch.linalg.cholesky(Zc)
        w = torch.cholesky_solve(torch.ones(n2, 1, dtype=torch.float64, device=Zc.device), L)
        torch.cuda.synchronize()
        ex["cusolver_fp64_n16384_s"] = time.perf_counter() - t0
        del L, w, Zc
    except Exception as e:  # noqa: BLE001
        ex["cusolver_fp64_error"] = str(e)[:120]
    # sweep on the grid-support cloud
    G = torch.from_numpy(workloads.grid_support_cloud()).cuda()
    t0 = time.perf_counter()
    r = ctx.sweep_tplus(G, 1e-3, 0.0, 1e-6)
    ex["sweep_grid_s"] = time.perf_counter() - t0
    ex["sweep_grid_tplus"] = r["t_plus"]
    ex["sweep_grid_probes"] = r["probes"]
    # gradients
    Xn = torch.from_numpy(workloads.normal_cloud()).cuda()
    t0 = time.perf_counter()
    ctx.grad(Xn, 2.0)
    torch.cuda.synchronize()
    ex["grad_n8192_m16_s"] = time.perf_counter() - t0
    # batch: 512 clouds in R^32 x 8 values of t (device-timed), and the same
    # problems one by one with the FP64 factor on a sample, for solves/s
    clouds, tvals = workloads.batch_clouds()
    cl = [torch.from_numpy(c).cuda() for c in clouds]
    ctx.set_options(M.Options())
    ctx.solve_batch(cl[:16], list(tvals))  # warm-up and tuner
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, _, sts = ctx.solve_batch(cl, list(tvals))
    e1.record()
    torch.cuda.synchronize()
    nsolves = len(cl) * len(tvals)
    ex["batch_solves"] = nsolves
    ex["batch_s"] = e0.elapsed_time(e1) / 1e3
    ex["batch_solves_per_s"] = nsolves / ex["batch_s"]
    ex["batch_failed"] = int((sts != 0).sum())
    ctx.set_options(M.Options(precision="fp64"))
    sample = [(c, t) for c in cl[::64] for t in tvals[::4]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, t in sample:
        ctx.solve(c, float(t))
    torch.cuda.synchronize()
    ex["per_instance_fp64_solves_per_s"] = len(sample) / (time.perf_counter() - t0)
    ex["per_instance_fp64_sample"] = f"{len(sample)} problems (every 64th cloud, t[0] and t[4])"
    # scale-zero weighting (App. C, Eq. scaleZero) on the precision config's
    # cloud (n = 16384) and on the headline cloud
    ctx.set_options(M.Options(precision=a.precision, residual_mode=a.resid))
    for name, Xs in (("mixture_n16384", Xm), ("cube_n%d" % Xd.shape[0], Xd)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, s0, i0 = ctx.scale_zero(Xs)
        torch.cuda.synchronize()
        ex[f"scale_zero_{name}_s"] = time.perf_counter() - t0
        ex[f"scale_zero_{name}_rel_residual"] = i0["rel_residual"]
        ex[f"scale_zero_{name}_ir_iters"] = i0["ir_iters"]
        ex[f"scale_zero_{name}_precision"] = i0["precision_used"]
    ctx.set_options(M.Options(precision=a.precision, residual_mode=a.resid, profile=True))
    out["extras"] = ex


# ---------------------------------------------------------- reference arm
def run_reference(a):
    import oracle
    import workloads
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    X = workloads.unit_cube_cloud(n=a.n, m=a.m)
    oracle.build()
    # size the sample so that all warm-up and timed steps take about 150 s:
    # time one 4096-point solve and scale by n^3 (between 2048 and the
    # --cpu-sample-n cap)
    Xc = workloads.subsample(X, min(4096, a.n), seed=12)
    t0 = time.perf_counter()
    oracle.weighting(Xc, 1.0, ir_steps=2)
    calib = time.perf_counter() - t0
    per_step = 150.0 / max(1, a.steps + a.warmup)
    n_s = int(Xc.shape[0] * (per_step / calib) ** (1.0 / 3.0)) // 256 * 256
    n_s = max(min(2048, a.n), min(n_s, a.cpu_sample_n, a.n))
    Xs = workloads.subsample(X, n_s, seed=11)
    times = []
    for k in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        oracle.weighting(Xs, 1.0, ir_steps=2)
        el = time.perf_counter() - t0
        if k >= a.warmup:
            times.append(el)
    tot = sum(times)
    flops = n_s ** 3 / 3 + 2 * n_s ** 2 * 2
    value = flops * len(times) / tot / 1e12
    sample = (f"each step: one oracle solve of a seeded {n_s}-point subset of the n={a.n}, m={a.m} "
              f"unit-cube workload at t=1 (Z, Cholesky, substitution, 2 FP64 refinement steps)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": tot / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"n={a.n} points uniform in [0,1]^{a.m}; bounded CPU sample n={n_s}",
                       "n": a.n, "m": a.m, "sample_n": n_s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch_only(a):
    """The batched solver alone: 512 clouds in R^32 (sizes log-uniform in
    [64, 2048]) x 8 values of t, one persistent launch; warm-up, then a
    device-timed run per step."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    torch.cuda.set_device(0)
    ctx = M.Context(M.Options())
    clouds, tvals = workloads.batch_clouds()
    cl = [torch.from_numpy(c).cuda() for c in clouds]
    for _ in range(max(1, a.warmup)):
        ctx.solve_batch(cl, list(tvals))
    torch.cuda.synchronize()
    times = []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, sts = ctx.solve_batch(cl, list(tvals))
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    nsolves = len(cl) * len(tvals)
    best = min(times)
    return {"metric": "batch solves per second (512 clouds in R^32 x 8 t, rel. residual <= 1e-14)",
            "value": nsolves / best, "unit": "solves/s", "seconds": times, "solves": nsolves,
            "failed": int((sts != 0).sum()), "data": "synthetic"}


def run_paper_sweep(a):
    """The paper's runtime workload: for every (n, m, covariance, run) the
    cutoff t_+ on [1e-3, bound] (rel. width 1e-6) and the weighting there, by
    bisection and by Ridders' method; wall time per sweep on one GPU."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = M.Context(M.Options(precision=a.precision, residual_mode=a.resid))
    # warm-up: library load, workspace, task tables
    ctx.sweep_tplus(torch.from_numpy(workloads.paper_runtime_cloud(1000, 3)).cuda(), 1e-3, 0.0, 1e-6)
    rows = []
    units = [(n, m, c, r) for n in workloads.PAPER_RUNTIME_NS for m in workloads.PAPER_RUNTIME_MS
             for c in workloads.PAPER_RUNTIME_COVS for r in range(3)]
    for i, (n, m, c, r) in enumerate(units):
        if i % world != rank:
            continue
        Xd = torch.from_numpy(workloads.paper_runtime_cloud(n, m, c, r)).cuda()
        for method in ("bisection", "ridders"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                res = ctx.sweep_tplus(Xd, 1e-3, 0.0, 1e-6, method=method)
                torch.cuda.synchronize()
                rows.append({"n": n, "m": m, "cov": c, "run": r, "method": method,
                             "seconds": time.perf_counter() - t0, "t_plus": res["t_plus"],
                             "bracket": list(res["bracket"]), "below": res["below"],
                             "probes": res["probes"], "mag": res["mag"],
                             "rel_residual": res["info"]["rel_residual"]})
            except M.MagnitudeError as e:
                rows.append({"n": n, "m": m, "cov": c, "run": r, "method": method, "status": e.status,
                             "error": str(e)[:160]})
    return {"metric": "paper runtime workload: t_+ and w(t_+) per point cloud", "unit": "s",
            "n_gpus": world, "rank": rank, "data": "synthetic", "rows": rows}


def run_fp64_dense_headline(a):
    """One solve of the headline workload's first t (points uniform in
    [0,1]^m, t = 1) by this library's plain FP64 path (precision = fp64) and
    by AUTO, device-timed, and optionally cuSOLVER's FP64 Cholesky on the full
    square matrix.  Minutes per FP64 solve at n = 1e5 (1.2 TFLOP/s FP64)."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = a.fp64_dense_n
    X = torch.from_numpy(workloads.unit_cube_cloud(n=n, m=a.m)).to(dev)
    sampler = ClockSampler(_gpu_id(dev))
    out = {"metric": "FP64 dense vs mixed+IR solve time", "n": n, "m": a.m, "t": 1.0, "data": "synthetic",
           "workload": f"n={n} points uniform in [0,1]^{a.m} (seed {workloads.SEEDS['cube']}), t=1"}
    sampler.start()
    for prec in ("auto", "fp64"):
        c = M.Context(M.Options(precision=prec, profile=True))
        if prec == "auto":
            c.solve(X, 1.0)  # warm-up (task tables, workspace)
        el, (_, mag, info) = _event_time(lambda: c.solve(X, 1.0), dev)
        out[prec] = {"seconds": el, "ms_generate": info["ms_generate"], "ms_factor": info["ms_factor"],
                     "ms_solve": info["ms_solve"], "ms_residual": info["ms_residual"],
                     "ir_iters": info["ir_iters"], "rel_residual": info["rel_residual"], "mag": mag,
                     "precision_used": info["precision_used"], "useful_flops": info["useful_flops"],
                     "tflops": info["useful_flops"] / el / 1e12}
        c.close()
        torch.cuda.empty_cache()
    if not a.no_cusolver:
        try:
            def cusolver():
                Z = torch.cdist(X, X).mul_(-1.0).exp_()
                torch.linalg.cholesky(Z, out=Z)  # in place: 8 n^2 bytes in all
                return torch.cholesky_solve(torch.ones(n, 1, dtype=torch.float64, device=dev), Z)
            el, _ = _event_time(cusolver, dev)
            out["cusolver_fp64"] = {"seconds": el, "tflops": (n ** 3 / 3) / el / 1e12}
        except Exception as e:  # noqa: BLE001
            out["cusolver_fp64"] = {"error": str(e)[:200]}
    out["clocks"] = sampler.stop()
    out["speedup_vs_own_fp64"] = out["fp64"]["seconds"] / out["auto"]["seconds"]
    return out


def run_out_of_core(a):
    """One solve of a workload past the GPU's memory (the packed FP32 tiles
    alone exceed it): the slabs, the bytes kept in host memory, the rate of
    the reads from host memory over the CPU-GPU link, and the solve's time."""
    import torch

    import paper_2607_23354_gb300 as M
    import workloads
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = a.ooc_n
    t = float(a.ts.split(",")[0])
    X = torch.from_numpy(workloads.unit_cube_cloud(n=n, m=a.m)).to(dev)
    c = M.Context(M.Options(profile=True))
    sampler = ClockSampler(_gpu_id(dev))
    sampler.start()
    el, (_, mag, info) = _event_time(lambda: c.solve(X, t), dev)
    clocks = sampler.stop()
    keys = ("precision_used", "probe_rho", "ir_iters", "gmres_iters", "fallback", "rel_residual", "slabs",
            "host_slabs", "host_bytes", "host_read_bytes", "ms_host_read", "ms_generate", "ms_factor", "ms_solve",
            "ms_residual", "residual_evals", "update_launches", "ms_update", "ms_update_busy", "update_flops",
            "useful_flops")
    out = {"metric": "solve beyond one GPU's memory (out-of-core factor)", "n": n, "m": a.m, "t": t,
           "data": "synthetic", "workload": f"n={n} points uniform in [0,1]^{a.m} (seed {workloads.SEEDS['cube']})",
           "fp32_tile_bytes": ((n + 127) // 128) * ((n + 127) // 128 + 1) // 2 * 128 * 128 * 4,
           "device_bytes": torch.cuda.get_device_properties(dev).total_memory,
           "seconds": el, "mag": mag, "tflops": info["useful_flops"] / el / 1e12,
           "info": {k: info[k] for k in keys}, "clocks": clocks}
    if info["ms_host_read"] > 0:
        out["host_read_gbs"] = info["host_read_bytes"] / (info["ms_host_read"] / 1e3) / 1e9
    if info["update_launches"]:
        busy = info["ms_update_busy"] or info["ms_update"]
        out["update_tflops"] = info["update_flops"] / (busy / 1e3) / 1e12 if busy else None
    c.close()
    return out


def main():
    a = parse_args()
    if a.ooc_n:
        print(json.dumps(run_out_of_core(a)), flush=True)
        return
    if a.fp64_dense_n:
        print(json.dumps(run_fp64_dense_headline(a)), flush=True)
        return
    if a.paper_sweep:
        print(json.dumps(run_paper_sweep(a)), flush=True)
        return
    if a.batch_only:
        print(json.dumps(run_batch_only(a)), flush=True)
        return
    if a.impl == "reference":
        out = run_reference(a)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out, state = run_ours(a)
    rank, world, _ = dist_env()
    if rank == 0:
        ctx, Xd, X, ts = state
        if not a.no_comparators:
            # the metric's other two parts, outside the timed region
            out["fp64_dense"] = fp64_dense_comparison(Xd.device)
            out["batch"] = batch_throughput(Xd.device)
            out["batch_solves_per_s"] = out["batch"]["solves_per_s"]
        if a.extras:
            run_extras(ctx, a, out, Xd)
        if not a.no_cpu:
            out["cpu_baseline"] = cpu_oracle_sample(X, 1.0, min(a.cpu_sample_n, a.n))
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

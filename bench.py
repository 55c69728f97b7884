"""Benchmark of the GB300 adaptive solver on the batched workload.

Workload (one "step" = one pass of the whole adaptive solve over one batch):
10,000 independent FP64 systems, n ~ U[16, 512], nrhs ~ U[1, 8], class mix
40% general N(0,1) + 2 sqrt(n) I, 25% SPD G^T G / n + I, 15% banded
(kl, ku ~ U[1, 16], diagonally dominant), 15% triangular (half upper, half
lower, diagonally dominant), 5% U diag(logspace(0, -13)) V^T with Haar U, V.
Every step scans, routes, factors, solves, estimates rcond, refines and
(when needed) runs the SVD fallback for all 10,000 systems.

metric: solves/s at backward error <= 1e-13 (systems whose in-kernel FP64
backward error is above 1e-13, or that took the approximate SVD route, are
not counted).  The plain FP64 GPU path (same pipeline, FP64 factorisations)
is timed beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) each rank solves its own batch (weak scaling).

More workloads print their own JSON line (not the headline):
  --workload large   single dense systems n in --sizes (default 8192,16384),
                     general U diag(logspace(0,-k)) V^T and SPD with kappa in
                     {1e2, 1e4, 1e6}, nrhs in {1, 64}: mixed precision
                     (FP32 factors on tcgen05, FP64 refinement) vs the FP64
                     path, time per solve with CUDA events.
  --workload band    one band system in band storage, n = 10^6, kl = ku in
                     {2, 8, 32}, nrhs in {1, 16}: time per asolve_solve_band.
  --workload plain   five single systems at n = 200 (general N(0,1), lower
                     triangular, SPD, tridiagonal, U diag(logspace(0,-14)) V^T
                     with Haar U, V), one right-hand side: latency of one
                     asolve_solve call per system over --reps repetitions.
  --workload replica the paper's Tables 1-4 on the GPU: 1000 random systems
                     per kind (5-diagonal band, lower triangular, sympd,
                     dense) and n in {100, 250, 500, 1000}, adaptive solver
                     vs the standard LU solver (ASOLVE_FORCE_LU), time per
                     system and reduction in %.
  --workload serve   request server: Poisson arrivals of FP64 requests in
                     host memory, n log-uniform in [32, 8192], the batched
                     class mix, kappa log-uniform in [1e1, 1e12], HBM budget
                     120 GB; capacity at saturation, then p50/p99 latency at
                     fractions of it.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s at backward err <=1e-13 (batched adaptive solve)"
UNIT = "solves/s"
WORKLOAD = "batched-10000: n~U[16,512], nrhs~U[1,8], mix 40% general/25% spd/15% banded/15% tri/5% ill"
BERR_BAR = 1e-13
# arithmetic peaks of one GB300: measured by the library's pipe probes
# (paper_2007_11208_gb300/peaks.py -> pipe_peaks.json); these defaults are
# that file's values, used only if it is missing
PIPE_PEAKS = os.path.join(ROOT, "paper_2007_11208_gb300", "pipe_peaks.json")
PEAK_FP32 = 78.46e12
PEAK_DFMA = 1.254e12
PEAK_DMMA = 1.095e12
COUNT = 10000  # systems per GPU per step (--count overrides, for small profiling runs)
# dram__bytes_read.sum + dram__bytes_write.sum of k_lu_class on the
# 1,000-system batch of the same generator (3.689203 GB + 1.292845 GB), from
# an ncu capture of the timed step of `bench.py --count 1000 --steps 1
# --warmup 1 --no-cpu-baseline`
LU_CLASS_DRAM_BYTES_1000 = 3.689203e9 + 1.292845e9
TUNING = os.path.join(ROOT, "paper_2007_11208_gb300", "tuning.json")  # autotuner output, if present
SEED = 1


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------- inputs
def make_batch(device, seed, count=COUNT):
    from paper_2007_11208_gb300 import synth
    specs = synth.batch_specs(count, seed)
    pk = synth.packed_batch(specs, seed + 1000, device=device)
    pk["specs"] = specs
    for k in ("n", "nrhs", "a_off", "b_off"):
        pk[k + "_h"] = pk[k].clone()
        pk[k] = pk[k].to(device)
    return pk


def algorithmic_bytes_scan(specs):
    return sum(8 * n * n + 8 * n * r for (_, n, r, *_rest) in specs)


# --------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


# --------------------------------------------------------------- our arm
def decode_infos(t):
    from paper_2007_11208_gb300 import asolve
    return asolve.infos_from_tensor(t)


def run_steps(ctx, pk, X, infos, flags, steps, stream):
    """Time `steps` batched solves with CUDA events on the context stream."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        ev0.record(stream)
        rc = ctx.solve_batched(COUNT, pk["n"], pk["nrhs"], pk["a_off"], pk["b_off"], pk["A"], pk["B"],
                               X, infos, flags)
        ev1.record(stream)
        torch.cuda.synchronize()
        assert rc == 0, rc
        times.append(ev0.elapsed_time(ev1))
    return times


def verified_count(infos_list):
    ok = 0
    hist = {}
    for i in infos_list:
        key = (i["route"], i["precision"], i["status"])
        hist[key] = hist.get(key, 0) + 1
        if i["status"] == 0 and i["berr"] == i["berr"] and i["berr"] <= BERR_BAR:
            ok += 1
    return ok, hist


def pipe_peaks():
    """FP32 FMA, FP64 FMA and FP64 mma.sync peaks (FLOP/s) and their source."""
    if os.path.exists(PIPE_PEAKS):
        d = json.load(open(PIPE_PEAKS))
        return (d["ffma_tflops"] * 1e12, d["dfma_tflops"] * 1e12, d["dmma_tflops"] * 1e12,
                "measured (pipe_peaks.json: asolve_pipe_peak probes)")
    return PEAK_FP32, PEAK_DFMA, PEAK_DMMA, "measured (defaults copied from pipe_peaks.json)"


# Triangular solves the 1-norm estimate takes per system (Hager/Higham:
# x = inv(A) e/n, a transposed solve, then usually one more pair, and the
# final alternating-sign vector): counted as 5 solves of 2 n^2 flops.
EST_SOLVES = 5


def flops_model(specs, infos_list):
    """Algorithmic arithmetic of the dense class kernels per step, split by
    the pipe it runs on, and the time floor it sets.

    Mixed route: FP32 factorisation (LU 2n^3/3, Cholesky n^3/3), FP32
    solves (2 n^2 nrhs per refinement step, the estimate's solves) and FP64
    residuals (2 n^2 nrhs per refinement step plus the converged check).
    FP64 route (rcond gate or stall): FP64 factorisation, solve, estimate
    and the backward-error residual.  The FP64 tensor instruction runs at
    the DFMA rate on this GPU (measured), so every FP64 flop is charged at
    the larger of the two measured FP64 rates; the floor of a kernel is the
    larger of its FP32 and FP64 times (the pipes run concurrently)."""
    p32, pdfma, pdmma, src = pipe_peaks()
    p64 = max(pdfma, pdmma)
    out = {"lu32": 0.0, "chol32": 0.0, "lu64": 0.0, "chol64": 0.0, "res64": 0.0}
    per = {"k_lu_class": [0.0, 0.0], "k_chol_class": [0.0, 0.0]}  # [fp32, fp64] flops
    for (kind, n, r, *_), inf in zip(specs, infos_list):
        route, prec, it = inf["route"], inf["precision"], inf["ir_iters"]
        kern = "k_lu_class" if route in (6, 5) else ("k_chol_class" if route == 4 else None)
        if kern is None:
            continue
        f = (2.0 / 3.0 if kern == "k_lu_class" else 1.0 / 3.0) * n ** 3
        solves = 2.0 * n * n * (r * (it + 1) + EST_SOLVES)
        if prec == 1:
            res = 2.0 * n * n * r * (it + 1)
            out["res64"] += res
            out["lu32" if kern == "k_lu_class" else "chol32"] += f
            per[kern][0] += f + solves
            per[kern][1] += res
        else:
            # a rejected FP32 attempt (gate) was paid for as well
            if inf["detail"] & 3:
                per[kern][0] += f + 2.0 * n * n * EST_SOLVES
            out["lu64" if kern == "k_lu_class" else "chol64"] += f
            res = 2.0 * n * n * r
            out["res64"] += res
            per[kern][1] += f + 2.0 * n * n * (r + EST_SOLVES) + res
    t_min = {k: max(v[0] / p32, v[1] / p64) * 1e3 for k, v in per.items()}
    out.update(t_min_ms=t_min, flops_fp32={k: v[0] for k, v in per.items()},
               flops_fp64={k: v[1] for k, v in per.items()},
               peaks_tflops={"fp32": p32 / 1e12, "fp64": p64 / 1e12}, peaks_src=src)
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


def large_case_roofline(kind, prec, n, nrhs, ms, peaks):
    """Roofline of one single-system solve: the larger of two time floors,
    the algorithmic flops at the peak of the arithmetic that bounds them and
    one read of A (8 n^2 bytes) at the HBM peak; frac = floor / measured.

    Flops: LU 2n^3/3, Cholesky n^3/3 (plus 2 n^2 nrhs for the two
    triangular solves), triangular route n^2 nrhs.  Peaks: the FP64 path and
    the triangular route at the FP64 pipe rate measured on this GPU (the
    larger of the DFMA and mma.sync f64 probes); the mixed path's trailing updates at the 3xTF32 rate
    (three TF32 products, TF32 = half the measured bf16 burst rate); the
    BF16 / FP16 updates at the measured bf16 burst rate; the Ozaki-split
    FP64 updates (FP64_OZ mode, and the triangular route's blocked updates
    from 32 right-hand sides in every mode but FP64) at the bf16 burst rate
    / 28, the slice products per FP64 product."""
    flops = {"general": 2.0 / 3.0 * n ** 3 + 2.0 * n * n * nrhs,
             "spd": 1.0 / 3.0 * n ** 3 + 2.0 * n * n * nrhs,
             "lower": float(n) * n * nrhs}[kind]
    bf16 = peaks["bf16_tflops"] * 1e12
    if prec == "fp64_oz" or (kind == "lower" and prec != "fp64" and nrhs >= 32):
        peak, unit_src = bf16 / 28.0, f"Ozaki split: bf16 {peaks['src']} / 28"
    elif kind == "lower" or prec == "fp64":
        p32, pdfma, pdmma, src = pipe_peaks()
        peak, unit_src = max(pdfma, pdmma), "FP64 pipe, " + src
    elif prec == "mixed":
        peak, unit_src = bf16 / 6.0, f"3xTF32 = bf16 {peaks['src']} / 6"
    elif prec == "fp8":
        peak, unit_src = 2.0 * bf16, f"FP8 = bf16 {peaks['src']} x 2 (nominal dense ratio 4.5 / 2.25)"
    else:
        peak, unit_src = bf16, f"bf16 {peaks['src']} (burst)"
    t_alu = flops / peak
    t_hbm = 8.0 * n * n / (peaks["hbm_gbs"] * 1e9)
    floor = max(t_alu, t_hbm)
    return {"bound": "alu" if t_alu >= t_hbm else "hbm", "flops": flops,
            "achieved_tflops": flops / (ms * 1e-3) / 1e12, "peak_tflops": peak / 1e12,
            "peak_src": unit_src, "floor_ms": floor * 1e3, "frac": floor / (ms * 1e-3)}


def oracle_solve_verified(oracle, A, B):
    """One system through the oracle, counted like the GPU arm counts it:
    status OK (no SVD route) and a backward error <= 1e-13 in every
    column, from the oracle's compensated residual."""
    X, inf = oracle.solve(A, B)
    if inf["status"] != 0:
        return False
    _, berr = oracle.residual_dot2(A, X, B)
    return bool(np.all(berr <= BERR_BAR))


def oracle_time_ms(fn, reps=1):
    """Median wall time of fn() in ms (the oracle on one host core)."""
    t = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        t.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(t)


def oracle_large_baseline(kinds, sizes, kappa=1e4, n0=2048):
    """The oracle on one n0 system per kind (same recipes as the large
    workload, CPU generator), extrapolated to each size by n^3 (n^2 for
    the triangular route): a naive O(n^3) solve at n = 16384 would take
    hours.  Returns {kind: {"measured_ms": ms at n0, "extrapolated_ms": {n: ms}}}."""
    import oracle
    from paper_2007_11208_gb300 import synth
    oracle.build()
    out = {}
    for kind in kinds:
        g = synth.gen(int(n0 + 17 * kappa) % 100003)
        if kind == "lower":
            M = synth.tri_dd(n0, g, lower=True)
        else:
            M = synth.spectrum_fast(n0, g, kappa, spd=(kind == "spd"))
        A = M.numpy().T
        b = synth.rhs(n0, 1, g).numpy().reshape(n0, 1)
        ms = oracle_time_ms(lambda: oracle.solve(A, b))
        p = 2 if kind == "lower" else 3
        out[kind] = {"measured_ms": ms, "n": n0,
                     "extrapolated_ms": {str(n): ms * (n / n0) ** p for n in sizes}}
    return out


def oracle_sample(pk, budget_s=15.0, max_threads=None):
    """Time the oracle as it stands on a bounded sample of the batch."""
    import oracle
    oracle.build()
    specs = pk["specs"]
    Ah = pk["A"].cpu().numpy()
    Bh = pk["B"].cpu().numpy()
    ao = pk["a_off_h"].numpy()
    bo = pk["b_off_h"].numpy()
    cores = max_threads or os.cpu_count() or 1
    # estimate cost ~ n^3 and pick a prefix of the batch worth ~budget_s
    order = list(range(len(specs)))
    # calibrate with a few systems
    def one(s):
        n, r = specs[s][1], specs[s][2]
        A = Ah[ao[s]:ao[s] + n * n].reshape(n, n).T
        B = Bh[bo[s]:bo[s] + n * r].reshape(r, n).T
        return oracle_solve_verified(oracle, A, B)
    t0 = time.perf_counter()
    cal = order[:8]
    for s in cal:
        one(s)
    t_cal = time.perf_counter() - t0
    per_n3 = t_cal / max(sum(specs[s][1] ** 3 for s in cal), 1)
    budget_work = budget_s * cores / max(per_n3, 1e-15)
    sample, acc = [], 0.0
    for s in order:
        acc += specs[s][1] ** 3
        sample.append(s)
        if acc >= budget_work:
            break
    import concurrent.futures as cf
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        oks = list(ex.map(one, sample))
    dt = time.perf_counter() - t0
    ok = sum(oks)
    return {"value": ok / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {len(sample)} of the {len(specs)} systems of the same batch "
                      f"(threads across systems), {dt:.1f} s"}


def aggregate_ranks(local_ms, local_ok, dist=None, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's time (max) and the
    verified systems of every rank (sum).  No data moves between ranks:
    each rank solves its own batch."""
    tt = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    okt = torch.tensor([float(local_ok)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.barrier()
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(okt, op=dist.ReduceOp.SUM)
    return tt.item(), okt.item()


def rank_seed(rank):
    """Seed of rank `rank`'s batch (independent systems per rank)."""
    return SEED + 7919 * rank


def ours(args):
    from paper_2007_11208_gb300 import asolve, build
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    pk = make_batch(dev, rank_seed(rank), COUNT)
    torch.cuda.synchronize()
    log(f"[rank {rank}] batch generated in {time.perf_counter() - t_gen:.1f}s; "
        f"A bytes {pk['A'].numel() * 8 / 1e9:.2f} GB")
    specs = pk["specs"]
    X = torch.zeros_like(pk["B"])
    infos = torch.zeros(COUNT * asolve.INFO_BYTES, dtype=torch.uint8, device=dev)
    flags = asolve.BERR

    def arm(precision, steps, warmup, profile=False):
        ctx = asolve.Context(precision=precision, tuning=TUNING if os.path.exists(TUNING) else None)
        stream = torch.cuda.ExternalStream(ctx.stream)
        run_steps(ctx, pk, X, infos, flags, warmup, stream)
        if profile:
            ctx.set_profiling(True)
            ctx.reset_profile()
        with ClockSampler(local) as clk:
            times = run_steps(ctx, pk, X, infos, flags, steps, stream)
        prof = ctx.profile() if profile else None
        inf_list = decode_infos(infos)
        ctx.close()
        return times, inf_list, clk.summary(), prof

    # headline: mixed precision path
    times, inf_mixed, clocks, _ = arm(asolve.PREC_MIXED, args.steps, args.warmup)
    ok, hist = verified_count(inf_mixed)
    total_ms, ok_all = aggregate_ranks(sum(times), ok, dist, dev)
    value = ok_all * args.steps / (total_ms / 1e3)
    if args.quick:
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "quick": True,
                          "ms_per_step": total_ms / args.steps, "count": COUNT}), flush=True)
        return
    # plain FP64 GPU path on the same batch
    t64, inf64, _, _ = arm(asolve.PREC_FP64, max(1, min(args.steps, 2)), 1)
    ok64, hist64 = verified_count(inf64)
    fp64_value = ok64 / (statistics.mean(t64) / 1e3)
    # per-kernel profile of the headline path (CUDA events around each launch)
    _, _, _, prof = arm(asolve.PREC_MIXED, args.steps, 1, profile=True)
    # e2e through the C ABI with host buffers (copies inside the timed region)
    e2e = e2e_arm(pk, args)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 factors + FP64 refinement)",
        "data": "synthetic (seeded; shapes and distributions of the batched configuration)",
        "config": {"workload": WORKLOAD, "systems_per_gpu": COUNT, "global_batch": COUNT * world,
                   "parallelism": f"replicas x{world}", "l2": "inputs (7.2 GB/GPU) larger than L2",
                   "precision": "mixed",
                   "panel_widths": "autotuned (tuning.json)" if os.path.exists(TUNING) else "built-in rule"},
        "verified_per_step": ok, "verified_fraction": ok / COUNT,
        "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_step": statistics.mean(t64),
                      "verified_per_step": ok64},
        "speedup_vs_fp64_path": value / max(fp64_value * world, 1e-30),
        "routes": {f"route{k[0]}_prec{k[1]}_st{k[2]}": v for k, v in sorted(hist.items())},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": 7 * args.steps,
    }
    # roofline of the dominant kernel
    peaks = load_peaks()
    if prof:
        per = {k: v[1] / max(v[0], 1) for k, v in prof.items() if v[0]}
        result["kernel_ms"] = per
        dom = max(per, key=per.get)
        fm = flops_model(specs, inf_mixed)
        if dom == "k_scan_batched":
            byt = algorithmic_bytes_scan(specs)
            ach = byt / (per[dom] / 1e3) / 1e9
            result["roofline"] = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                                  "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
                                  "peak_src": peaks["src"]}
        else:
            # the class kernels are bound by their arithmetic: the FP64 pipe
            # (residuals, FP64 factorisations) is the scarcer of the two
            f64 = fm["flops_fp64"].get(dom, 0.0)
            f32 = fm["flops_fp32"].get(dom, 0.0)
            p64 = fm["peaks_tflops"]["fp64"]
            p32 = fm["peaks_tflops"]["fp32"]
            sec = per[dom] / 1e3
            ach = f64 / sec / 1e12
            traffic = None
            if dom == "k_lu_class" and COUNT > 0:
                # DRAM bytes (read + write) of one k_lu_class launch from an ncu
                # capture of a 1,000-system batch of the same generator,
                # scaled by the number of systems
                traffic = LU_CLASS_DRAM_BYTES_1000 * COUNT / 1000.0
            t_min = fm["t_min_ms"].get(dom, 0.0)
            result["roofline"] = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": p64,
                                  "unit": "TFLOP/s", "frac": ach / p64, "traffic": traffic,
                                  "traffic_unit": "bytes per launch",
                                  "peak_src": "FP64 pipe, " + fm["peaks_src"],
                                  "fp32": {"flops": f32, "achieved": f32 / sec / 1e12, "peak": p32,
                                           "frac": f32 / sec / 1e12 / p32},
                                  "fp64_flops": f64,
                                  "alu_time_model": {"min_ms": t_min, "measured_ms": per[dom],
                                                     "frac": t_min / per[dom]}}
        result["flops_model"] = fm
    if rank == 0 and args.cpu_baseline:
        result["cpu_baseline"] = oracle_sample(pk, budget_s=args.cpu_seconds)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def e2e_arm(pk, args):
    """Same metric through the C ABI with host buffers: per step the H2D copy
    of A, B and the metadata, the solve, and the D2H copy of X and the infos
    are inside the timed region."""
    from paper_2007_11208_gb300 import asolve
    Ah = pk["A"].cpu().pin_memory()
    Bh = pk["B"].cpu().pin_memory()
    Xh = torch.zeros_like(Bh).pin_memory()
    meta = [pk[k + "_h"].contiguous() for k in ("n", "nrhs", "a_off", "b_off")]
    infos = torch.zeros(COUNT * asolve.INFO_BYTES, dtype=torch.uint8).pin_memory()
    ctx = asolve.Context(precision=asolve.PREC_MIXED)
    flags = asolve.BERR | asolve.HOST_BUFFERS
    call = lambda: ctx.solve_batched(COUNT, meta[0].data_ptr(), meta[1].data_ptr(), meta[2].data_ptr(),
                                     meta[3].data_ptr(), Ah.data_ptr(), Bh.data_ptr(), Xh.data_ptr(),
                                     infos.data_ptr(), flags)
    for _ in range(max(1, args.warmup)):
        assert call() == 0
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        assert call() == 0
        t.append(time.perf_counter() - t0)
    ok, _ = verified_count(asolve.infos_from_tensor(infos))
    ctx.close()
    h2d = Ah.numel() * 8 + Bh.numel() * 8 + 4 * COUNT * 8
    d2h = Xh.numel() * 8 + COUNT * asolve.INFO_BYTES
    return {"value": ok / statistics.mean(t), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(t) * 1e3}


# ---------------------------------------------------------- reference arm
def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    from paper_2007_11208_gb300 import synth
    specs = synth.batch_specs(COUNT, SEED)
    pk = synth.packed_batch(specs[:400], SEED + 1000, device="cpu")
    cores = os.cpu_count() or 1
    Ah, Bh = pk["A"].numpy(), pk["B"].numpy()
    ao, bo = pk["a_off"].numpy(), pk["b_off"].numpy()
    sub = specs[:400]
    # sample size so a step takes ~budget seconds
    budget = max(2.0, min(args.cpu_seconds, 120.0 / max(args.steps + args.warmup, 1)))

    def one(s):
        n, r = sub[s][1], sub[s][2]
        A = Ah[ao[s]:ao[s] + n * n].reshape(n, n).T
        B = Bh[bo[s]:bo[s] + n * r].reshape(r, n).T
        return oracle_solve_verified(oracle, A, B)

    import concurrent.futures as cf
    t0 = time.perf_counter()
    one(0)
    per = (time.perf_counter() - t0) / max(sub[0][1] ** 3, 1)
    work, m = 0.0, 0
    while m < len(sub) and work < budget * cores / max(per, 1e-15):
        work += sub[m][1] ** 3
        m += 1
    vals, dts = [], []
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oks = list(ex.map(one, range(m)))
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                vals.append(sum(oks) / dt)
                dts.append(dt)
    v = statistics.mean(vals)
    sample = f"first {m} systems of the batched workload per step, threads across systems"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                      "higher_is_better": True, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(dts) * 1e3,
                      "scaling": "weak", "vs_baseline": None,
                      "config": {"workload": WORKLOAD, "systems_per_step": m},
                      "data": "synthetic", "dtype": "f64",
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


# --------------------------------------------------------------- large dense
def large_workload(args):
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sizes = [int(x) for x in args.sizes.split(",")]
    kappas = [float(x) for x in args.kappas.split(",")]
    kinds = args.kinds.split(",")
    nrhs_list = [int(x) for x in args.nrhs_list.split(",")]
    precs = [(asolve.PREC_MIXED, "mixed"), (asolve.PREC_FP64, "fp64"), (asolve.PREC_BF16, "bf16"),
             (asolve.PREC_FP16, "fp16"), (asolve.PREC_FP64_OZ, "fp64_oz"), (asolve.PREC_FP8, "fp8")]
    precs = [p for p in precs if p[1] in args.precs.split(",")]
    ctxs = {p: asolve.Context(precision=p) for p, _ in precs}
    peaks = load_peaks()
    cases = []
    with ClockSampler(0) as clk:
        for n in sizes:
            for kind in kinds:
                for kappa in kappas:
                    g = synth.gen(int(n + 17 * kappa) % 100003, dev)
                    if kind == "lower":  # TRSM: diagonally dominant lower triangle (kappa not imposed)
                        A = synth.tri_dd(n, g, lower=True, device=dev)
                    else:
                        A = synth.spectrum_fast(n, g, kappa, spd=(kind == "spd"), device=dev)
                    B64 = synth.rhs(n, max(nrhs_list), g, dev)
                    for nrhs in nrhs_list:
                        B = B64[:nrhs].contiguous()
                        X = torch.zeros_like(B)
                        row = {"n": n, "kind": kind, "kappa": kappa, "nrhs": nrhs}
                        for p, name in precs:
                            c = ctxs[p]
                            st = torch.cuda.ExternalStream(c.stream)
                            rc, info = c.solve(A, B, n, nrhs, X, asolve.BERR)  # warm-up (workspace)
                            times = []
                            for _ in range(args.steps):
                                e0 = torch.cuda.Event(enable_timing=True)
                                e1 = torch.cuda.Event(enable_timing=True)
                                torch.cuda.synchronize()
                                e0.record(st)
                                rc, info = c.solve(A, B, n, nrhs, X, asolve.BERR)
                                e1.record(st)
                                torch.cuda.synchronize()
                                times.append(e0.elapsed_time(e1))
                            ms = statistics.median(times)
                            row[name] = {"ms": ms, "rc": rc, "route": info["route"],
                                         "precision": info["precision"], "ir_iters": info["ir_iters"],
                                         "berr": info["berr"], "rcond": info["rcond"],
                                         "detail": info["detail"],
                                         "flops_per_s": ({"general": 2.0 / 3.0 * n ** 3, "spd": 1.0 / 3.0 * n ** 3,
                                                          "lower": float(n) * n * nrhs}[kind]) / (ms * 1e-3),
                                         "roofline": large_case_roofline(kind, name, n, nrhs, ms, peaks)}
                            log(n, kind, f"{kappa:.0e}", nrhs, name, f"{ms:.2f} ms", info["route"],
                                info["precision"], info["ir_iters"], f"{info['berr']:.2e}")
                        if "fp64" in row and "mixed" in row:
                            row["speedup"] = row["fp64"]["ms"] / row["mixed"]["ms"]
                        cases.append(row)
                    del A, B64
                    torch.cuda.empty_cache()
    for c in ctxs.values():
        c.close()
    head = [c for c in cases if c["n"] == sizes[-1] and c["kind"] == "general" and c["kappa"] == 1e4
            and c["nrhs"] == 1]
    head = head[0] if head else cases[-1]
    hp = next(p for p in ("mixed", "fp64", "fp64_oz", "bf16", "fp16", "fp8") if p in head)
    ok = head[hp]["rc"] == 0 and head[hp]["berr"] <= BERR_BAR
    cpu = None
    if args.cpu_baseline:
        ob = oracle_large_baseline(kinds, sizes)
        hk = ob.get(head["kind"])
        cpu = {"value": 1000.0 / hk["extrapolated_ms"][str(head["n"])] if hk else None, "unit": "solves/s",
               "cores": 1, "kind": "oracle",
               "sample": "one n = 2048 system per kind on one host core (nrhs 1), extrapolated by n^3 "
                         "(n^2 for the triangular route) to each size",
               "per_kind": ob}
    print(json.dumps({
        "metric": "solves/s at backward err <=1e-13 (single large dense system)",
        "value": (1000.0 / head[hp]["ms"]) if ok else 0.0, "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": head[hp]["ms"],
        "higher_is_better": True, "scaling": "replicas only", "vs_baseline": None,
        "dtype": "f64 (FP32 factors on tcgen05 3xTF32 + FP64 refinement)", "data": "synthetic",
        "config": {"workload": f"large-dense: {head['kind']} U diag(logspace(0,-k)) V^T, n={head['n']}, "
                               f"kappa={head['kappa']:.0e}, nrhs={head['nrhs']}, {hp}",
                   "l2": "inputs larger than L2"},
        "fp64_path_ms": head.get("fp64", {}).get("ms"), "speedup_vs_fp64_path": head.get("speedup"),
        "roofline": head[hp].get("roofline"), "cpu_baseline": cpu,
        "clocks": clk.summary(), "cases": cases}), flush=True)


# --------------------------------------------------------------- band
def band_workload(args):
    """Memory-bound configuration: one band system of order n = 10^6 in
    band storage, kl = ku = k, off-diagonal N(0,1), diagonal 1 + row abs
    sum, nrhs right-hand sides; time of one asolve_solve_band call (scan of
    the band, GBTRF-equivalent factorisation, solve, rcond estimate,
    backward error) with CUDA events."""
    if args.band_gbtrf_only:  # read by the library at its first band solve
        os.environ["ASOLVE_BAND_SPIKE"] = "0"
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = args.band_n
    ks = [int(x) for x in args.band_k.split(",")]
    nrhs_list = [int(x) for x in args.band_nrhs.split(",")]
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    ctx = asolve.Context()
    st = torch.cuda.ExternalStream(ctx.stream)
    rows, cpu_ms = [], {}
    with ClockSampler(0) as clk:
        for k in ks:
            g = synth.gen(1000 + k, dev)
            AB = synth.band_storage_dd(n, k, k, g, device=dev)  # row j = column j of the band layout
            Bm = synth.rhs(n, max(nrhs_list), g, dev)
            for nrhs in nrhs_list:
                B = Bm[:nrhs].contiguous()
                X = torch.zeros_like(B)
                rc, info = ctx.solve_band(AB, 2 * k + 1, k, k, B, n, nrhs, X, asolve.BERR)  # warm-up
                times = []
                for _ in range(args.steps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(st)
                    rc, info = ctx.solve_band(AB, 2 * k + 1, k, k, B, n, nrhs, X, asolve.BERR)
                    e1.record(st)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = statistics.median(times)
                io_bytes = 8.0 * n * (2 * k + 1) + 16.0 * n * nrhs  # band of A, B, X: each once
                row = {"n": n, "kl": k, "ku": k, "nrhs": nrhs, "ms": ms, "rc": rc, "route": info["route"],
                       "partitioned": bool(info["detail"] & 16),
                       "kl_found": info["kl"], "ku_found": info["ku"], "berr": info["berr"],
                       "rcond": info["rcond"], "io_bytes": io_bytes,
                       "io_gbs": io_bytes / (ms * 1e-3) / 1e9}
                row["io_frac_of_hbm"] = row["io_gbs"] / hbm
                rows.append(row)
                log(f"band n={n} k={k} nrhs={nrhs}: {ms:.2f} ms rc={rc} berr={info['berr']:.2e} "
                    f"A+B+X at {row['io_gbs']:.1f} GB/s")
            if args.cpu_baseline:  # the oracle on the same system, one right-hand side, one host core
                import oracle
                oracle.build()
                ABh = np.asfortranarray(AB.cpu().numpy().T)  # LAPACK layout (2k+1, n)
                bh = Bm[0].cpu().numpy().copy()
                cpu_ms[k] = oracle_time_ms(lambda: oracle.solve_band(ABh, k, k, bh))
                log(f"band n={n} k={k}: oracle {cpu_ms[k]:.0f} ms")
                del ABh
            del AB, Bm
            torch.cuda.empty_cache()
    ctx.close()
    head = rows[0]
    ok = all(r["rc"] == 0 and r["berr"] <= BERR_BAR for r in rows)
    print(json.dumps({
        "metric": "solves/s at backward err <=1e-13 (band system, n = 10^6)",
        "value": (1000.0 / head["ms"]) if ok else 0.0, "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "ms_per_step": head["ms"], "higher_is_better": True,
        "scaling": "replicas only", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"band: n={n}, kl=ku in {ks}, nrhs in {nrhs_list}, diagonally dominant, "
                               "band storage" + (", partitioned route off" if args.band_gbtrf_only else ""),
                   "l2": "inputs larger than L2"},
        "cpu_baseline": ({"value": 1000.0 / cpu_ms[ks[0]], "unit": "solves/s", "cores": 1, "kind": "oracle",
                          "sample": "one solve of the same system per k, one right-hand side, one host core",
                          "ms_per_k": {str(k): v for k, v in cpu_ms.items()}} if cpu_ms else None),
        "roofline_note": "the band factorisation is a sequential chain along n; io_gbs is the band of A, "
                         "B and X read or written once over the whole call, against the measured HBM copy "
                         "bandwidth",
        "clocks": clk.summary(), "cases": rows}), flush=True)


# --------------------------------------------------------------- plain
def launch_floor_us(reps=200):
    """Median host wall time of replaying a CUDA graph of one tiny kernel
    and synchronising: the floor under one asolve_solve call, which is one
    graph launch and one stream synchronisation.  None if the capture
    fails (the workload's own numbers stand without it)."""
    try:
        s = torch.cuda.Stream()
        x = torch.zeros(1, device="cuda")
        with torch.cuda.stream(s):
            x.add_(1.0)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
        for _ in range(20):
            g.replay()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            t0 = time.perf_counter()
            g.replay()
            torch.cuda.synchronize()
            t.append((time.perf_counter() - t0) * 1e6)
        return float(np.percentile(t, 50))
    except Exception as e:  # noqa: BLE001 -- a missing floor must not stop the workload
        log("launch floor not measured:", repr(e))
        return None


def plain_workload(args):
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = 200
    g = synth.gen(0, dev)
    mats = {"general": synth.general(n, g, dev), "lower": synth.lower_tri(n, g, dev),
            "spd": synth.spd(n, g, dev), "tridiag": synth.tridiag(n, g, dev),
            "ill": synth.ill(n, g, k=14.0, device=dev)}
    b = synth.rhs(n, 1, g, dev)
    ctx = asolve.Context()
    st = torch.cuda.ExternalStream(ctx.stream)
    x = torch.zeros_like(b)
    hb = b.cpu().pin_memory()
    hx = torch.zeros_like(hb).pin_memory()
    rows = []
    with ClockSampler(0) as clk:
        for name, A in mats.items():
            hA = A.cpu().pin_memory()
            for _ in range(20):
                ctx.solve(A, b, n, 1, x, 0)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.reps)]
            wall = []
            for e0, e1 in ev:
                t0 = time.perf_counter()
                e0.record(st)
                rc, info = ctx.solve(A, b, n, 1, x, 0)
                e1.record(st)
                wall.append((time.perf_counter() - t0) * 1e6)
            torch.cuda.synchronize()
            dev_us = np.array([e0.elapsed_time(e1) * 1e3 for e0, e1 in ev])
            e2e = []
            for _ in range(min(args.reps, 200)):
                t0 = time.perf_counter()
                ctx.solve(hA.data_ptr(), hb.data_ptr(), n, 1, hx.data_ptr(), asolve.HOST_BUFFERS)
                e2e.append((time.perf_counter() - t0) * 1e6)
            rows.append({"system": name, "route": info["route"], "status": rc, "rcond": info["rcond"],
                         "p50_us": float(np.percentile(wall, 50)), "p99_us": float(np.percentile(wall, 99)),
                         "device_p50_us": float(np.percentile(dev_us, 50)),
                         "e2e_p50_us": float(np.percentile(e2e, 50))})
            log(rows[-1])
    ctx.close()
    floor = launch_floor_us()
    cpu = None
    if args.cpu_baseline:  # the oracle on the same five systems, one host core
        import oracle
        oracle.build()
        bh = b.cpu().numpy().reshape(n, 1)
        per = {name: oracle_time_ms(lambda A=A: oracle.solve(A.cpu().numpy().T, bh), reps=20) * 1e3
               for name, A in mats.items()}
        cpu = {"value": float(np.median(list(per.values()))), "unit": "us", "cores": 1, "kind": "oracle",
               "sample": "the same five systems, 20 solves each, median", "per_system_us": per}
    med = float(np.median([r["p50_us"] for r in rows]))
    print(json.dumps({
        "metric": "latency of one adaptive solve (n=200, 1 rhs), median over the five systems",
        "value": med, "unit": "us", "n_gpus": 1, "steps": args.reps, "warmup": 20, "ms_per_step": med / 1e3,
        "higher_is_better": False, "scaling": "replicas only", "vs_baseline": None, "dtype": "f64 (mixed)",
        "data": "synthetic", "config": {"workload": "plain-200: general/lower/spd/tridiag/ill, seed 0"},
        "launch_floor_us": floor, "cpu_baseline": cpu,
        "e2e": {"value": float(np.median([r["e2e_p50_us"] for r in rows])), "unit": "us",
                "h2d_bytes_per_step": 8 * (n * n + n), "d2h_bytes_per_step": 8 * n + 64},
        "clocks": clk.summary(), "systems": rows}), flush=True)


# --------------------------------------------------------------- paper replica
# reduction (%) of the adaptive solver against the standard LU solver in the
# paper's Tables 1-3 (banded, triangular, sympd) and the detection overhead
# (%) of Table 4 (dense), n = 100, 250, 500, 1000; Intel Core i5-5200U
PAPER_TABLES = {"band5": [67.89, 83.45, 89.02, 91.18], "lower": [72.78, 73.59, 79.61, 84.09],
                "sympd": [17.35, 25.62, 24.02, 27.54], "dense": [-1.627, -0.243, -0.114, -0.187]}


def oracle_replica_tables(sizes=(100, 250, 500, 1000), count=4):
    """The paper's comparison with the oracle on one host core: the
    adaptive solve against the forced-LU solve, `count` systems per kind
    and n (the replica recipes, CPU generator), mean time per system."""
    import oracle
    from paper_2007_11208_gb300 import synth
    oracle.build()
    out = {}
    for kind in synth.REPLICA_KINDS:
        rows = []
        for n in sizes:
            pk = synth.replica_batch(kind, n, count, SEED + n)
            mats = []
            for s_ in range(count):
                o, q = int(pk["a_off"][s_]), int(pk["b_off"][s_])
                mats.append((pk["A"][o:o + n * n].numpy().reshape(n, n).T, pk["B"][q:q + n].numpy().copy()))
            t = {}
            for name, flags in (("standard", oracle.FORCE_LU), ("adaptive", 0)):
                t0 = time.perf_counter()
                for A, b in mats:
                    oracle.solve(A, b, flags=flags)
                t[name] = (time.perf_counter() - t0) / count
            rows.append({"n": n, "standard_s": t["standard"], "adaptive_s": t["adaptive"],
                         "reduction_pct": 100.0 * (1.0 - t["adaptive"] / t["standard"])})
        out[kind] = rows
    return out


def replica_workload(args):
    """The paper's evaluation (Sec. 3, Tables 1-4) on the GPU.  For each
    matrix kind and n, one batch of --replica-count random systems (one
    right-hand side each) is solved by the adaptive solver and by the
    standard solver (ASOLVE_FORCE_LU: LU whatever the structure; the scan
    still runs, for the non-finite check); time per system = batched call
    time / count, CUDA events on the context stream, median of --steps."""
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sizes = [int(x) for x in args.replica_sizes.split(",")]
    count = args.replica_count
    prec = {"fp64": asolve.PREC_FP64, "mixed": asolve.PREC_MIXED}[args.replica_prec]
    ctx = asolve.Context(precision=prec)
    st = torch.cuda.ExternalStream(ctx.stream)
    tables, launches = {}, 0
    with ClockSampler(0) as clk:
        for kind in synth.REPLICA_KINDS:
            rows = []
            for n in sizes:
                pk = synth.replica_batch(kind, n, count, SEED + n, dev)
                nd, rd = pk["n"].to(dev), pk["nrhs"].to(dev)
                ao, bo = pk["a_off"].to(dev), pk["b_off"].to(dev)
                X = torch.zeros_like(pk["B"])
                infos = torch.zeros(count * asolve.INFO_BYTES, dtype=torch.uint8, device=dev)
                row = {"n": n}
                for name, flags in (("standard", asolve.FORCE_LU), ("adaptive", 0)):
                    for _ in range(max(args.warmup, 1)):
                        rc = ctx.solve_batched(count, nd, rd, ao, bo, pk["A"], pk["B"], X, infos, flags)
                        assert rc == 0, rc
                    times = []
                    for _ in range(args.steps):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        torch.cuda.synchronize()
                        e0.record(st)
                        rc = ctx.solve_batched(count, nd, rd, ao, bo, pk["A"], pk["B"], X, infos, flags)
                        e1.record(st)
                        torch.cuda.synchronize()
                        assert rc == 0, rc
                        times.append(e0.elapsed_time(e1))
                        launches += 7
                    inf = asolve.infos_from_tensor(infos)
                    hist = {}
                    for i in inf:
                        hist[i["route"]] = hist.get(i["route"], 0) + 1
                    row[name] = {"s_per_system": statistics.median(times) * 1e-3 / count,
                                 "status_ok": sum(1 for i in inf if i["status"] == 0),
                                 "routes": {str(r): c for r, c in sorted(hist.items())}}
                a, b = row["adaptive"]["s_per_system"], row["standard"]["s_per_system"]
                row["reduction_pct"] = 100.0 * (1.0 - a / b)
                paper = dict(zip((100, 250, 500, 1000), PAPER_TABLES[kind])).get(n)
                if paper is not None:
                    row["paper_reduction_pct"] = paper
                log(kind, n, f"standard {b * 1e6:.1f} us", f"adaptive {a * 1e6:.1f} us",
                    f"reduction {row['reduction_pct']:.1f}%")
                rows.append(row)
                del pk, X, infos
                torch.cuda.empty_cache()
            tables[kind] = rows
    ctx.close()
    # headline of this workload: the mean reduction over the structured kinds
    red = [r["reduction_pct"] for kd in ("band5", "lower", "sympd") for r in tables[kd]]
    print(json.dumps({
        "metric": "reduction of time per system, adaptive vs standard LU (paper Tables 1-3)",
        "value": statistics.mean(red), "unit": "%", "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 1), "ms_per_step": None, "higher_is_better": True,
        "scaling": "replicas only", "vs_baseline": None,
        "dtype": "f64" if args.replica_prec == "fp64" else "f64 (mixed)", "data": "synthetic",
        "config": {"workload": f"paper-replica: {count} systems per kind and n, n in {sizes}, "
                               "band5/lower/sympd/dense (Sec. 3, Fig. 3 recipes), 1 rhs",
                   "l2": "inputs larger than L2 from n = 250 (count = 1000)"},
        "gpu_launches": launches, "clocks": clk.summary(), "tables": tables,
        "cpu_baseline": ({"kind": "oracle", "cores": 1, "sample": "4 systems per kind and n in {100, 250, 500, 1000}",
                          "tables": oracle_replica_tables()} if args.cpu_baseline else None)}), flush=True)


# --------------------------------------------------------------- serving
def _serve_templates(count, seed, dev, nmin=32, nmax=8192):
    """Request templates: n log-uniform, batched class mix, kappa log-uniform."""
    from paper_2007_11208_gb300 import synth
    g = synth.gen(seed, dev)
    gc = synth.gen(seed)
    out = []
    for t in range(count):
        u = torch.rand(4, generator=gc, dtype=torch.float64).tolist()
        n = int(round(math.exp(math.log(nmin) + u[0] * (math.log(nmax) - math.log(nmin)))))
        kappa = 10.0 ** (1.0 + 11.0 * u[1])
        nrhs = 1 + int(u[2] * 8) % 8
        if u[3] < 0.45:
            kind, M = "general", synth.spectrum_fast(n, g, kappa, device=dev)
        elif u[3] < 0.70:
            kind, M = "spd", synth.spectrum_fast(n, g, kappa, spd=True, device=dev)
        elif u[3] < 0.85:
            kl = 1 + int(u[0] * 1e6) % 16
            ku = 1 + int(u[1] * 1e6) % 16
            kind, M = "banded", synth.banded_kappa(n, kl, ku, g, kappa, device=dev)
        else:
            lower = int(u[2] * 1e6) % 2 == 0
            kind, M = "tri", synth.tri_kappa(n, g, kappa, lower=lower, device=dev)
        B = synth.rhs(n, nrhs, g, dev)
        out.append({"kind": kind, "n": n, "nrhs": nrhs, "kappa": kappa,
                    "A": M.cpu().pin_memory(), "B": B.cpu().pin_memory()})
        del M, B
    torch.cuda.empty_cache()
    return out


def serve_workload(args):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    tm = _serve_templates(args.templates, SEED + 5, dev)
    log(f"{len(tm)} templates in {time.perf_counter() - t0:.1f}s; "
        f"host bytes {sum(t['A'].numel() for t in tm) * 8 / 1e9:.2f} GB; "
        f"n: {sorted(t['n'] for t in tm)}")
    rng = np.random.default_rng(SEED + 6)
    R = args.requests
    pick = rng.integers(0, len(tm), size=R)
    Xs = [torch.zeros_like(tm[k]["B"]).pin_memory() for k in pick]
    flags = asolve.HOST_BUFFERS | asolve.BERR
    ctx = asolve.Context(hbm_budget=120 << 30)
    # warm the server (graphs, pools, workspaces) on every template once
    for k in range(len(tm)):
        t = tm[k]
        Xw = torch.zeros_like(t["B"])
        rc, tk = ctx.submit(t["A"].data_ptr(), t["B"].data_ptr(), t["n"], t["nrhs"], Xw.data_ptr(), flags)
        assert rc == 0
        ctx.poll(tk, -1)

    def run(rate):
        """Submit R requests with exponential gaps (rate <= 0: all at once)."""
        gaps = rng.exponential(1.0 / rate, size=R) if rate > 0 else np.zeros(R)
        before = ctx.serve_stats()
        tickets = []
        tstart = time.perf_counter()
        due = tstart
        for i, k in enumerate(pick):
            due += gaps[i]
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            t = tm[k]
            rc, tk = ctx.submit(t["A"].data_ptr(), t["B"].data_ptr(), t["n"], t["nrhs"],
                                Xs[i].data_ptr(), flags)
            assert rc == 0, rc
            tickets.append(tk)
        lat, ok, infos, missed = [], 0, [], {}
        for i, tk in enumerate(tickets):
            st, info, l = ctx.poll(tk, -1)
            lat.append(l)
            infos.append(info)
            if st == 0 and info["berr"] <= BERR_BAR:
                ok += 1
            else:  # which templates fall short of the bar, and how
                t, info = tm[pick[i]], info or {}
                missed.setdefault(int(pick[i]), {"kind": t["kind"], "n": t["n"], "kappa": t["kappa"],
                                                 "status": st, "route": info.get("route"),
                                                 "berr": info.get("berr"), "rcond": info.get("rcond"),
                                                 "count": 0})
                missed[int(pick[i])]["count"] += 1
        after = ctx.serve_stats()
        wall = time.perf_counter() - tstart
        busy = after["busy_ms"] - before["busy_ms"]
        lat = np.array(lat)
        return {"rate": rate, "requests": R, "wall_s": wall, "solves_per_s": ok / wall,
                "completed_per_s": R / wall, "verified": ok,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "busy_frac": busy / (wall * 1e3),
                "rounds": after["rounds"] - before["rounds"],
                "batches": after["batches"] - before["batches"],
                "large": after["large_solves"] - before["large_solves"],
                "peak_charged_gb": after["peak_charged_bytes"] / 1e9,
                "unverified": list(missed.values())}

    points = []
    with ClockSampler(0) as clk:
        sat = run(0.0)
        log("saturation", sat)
        points.append(sat)
        cap = sat["completed_per_s"]
        for f in [float(x) for x in args.load.split(",")]:
            p = run(f * cap)
            p["load"] = f
            log("load", f, p)
            points.append(p)
    ctx.close()
    h2d = sum(8 * (tm[k]["n"] ** 2 + tm[k]["n"] * tm[k]["nrhs"]) for k in pick)
    d2h = sum(8 * tm[k]["n"] * tm[k]["nrhs"] for k in pick)
    print(json.dumps({
        "metric": "solves/s at backward err <=1e-13 (request server, saturated)",
        "value": sat["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": sat["wall_s"] * 1e3, "higher_is_better": True, "scaling": "replicas only",
        "vs_baseline": None, "dtype": "f64 (mixed: FP32 factors + FP64 refinement)",
        "data": "synthetic",
        "config": {"workload": f"serve: {R} requests from {len(tm)} templates, n log-uniform [32,8192], "
                               "batched class mix, kappa log-uniform [1e1,1e12], host FP64 in/out, "
                               "HBM budget 120 GB"},
        "e2e": {"value": sat["solves_per_s"], "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"], "busy_frac": sat["busy_frac"],
        "clocks": clk.summary(), "points": points}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--count", type=int, default=COUNT,
                    help="systems per GPU (smaller values are for profiling runs only)")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "large", "serve", "plain", "band", "replica"])
    ap.add_argument("--band-gbtrf-only", action="store_true",
                    help="band: turn the partitioned route for dominant bands off (ASOLVE_BAND_SPIKE=0)")
    ap.add_argument("--replica-sizes", default="100,250,500,1000")
    ap.add_argument("--replica-count", type=int, default=1000)
    ap.add_argument("--replica-prec", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--band-n", type=int, default=1_000_000, help="band: order")
    ap.add_argument("--band-k", default="2,8,32", help="band: kl = ku values")
    ap.add_argument("--band-nrhs", default="1,16", help="band: right-hand-side counts")
    ap.add_argument("--reps", type=int, default=1000, help="plain: repetitions per system")
    ap.add_argument("--sizes", default="8192,16384", help="large: matrix sizes")
    ap.add_argument("--kinds", default="general,spd", help="large: matrix kinds (general, spd, lower)")
    ap.add_argument("--kappas", default="1e2,1e4,1e6", help="large: condition numbers")
    ap.add_argument("--nrhs-list", default="1,64", help="large: right-hand-side counts")
    ap.add_argument("--precs", default="mixed,fp64", help="large: precisions (mixed, fp64, bf16, fp16, fp64_oz, fp8)")
    ap.add_argument("--templates", type=int, default=40, help="serve: distinct request matrices")
    ap.add_argument("--requests", type=int, default=160, help="serve: requests per load point")
    ap.add_argument("--load", default="0.25,0.5,0.8", help="serve: arrival rates as fractions of capacity")
    ap.add_argument("--quick", action="store_true",
                    help="headline arm only (no FP64 comparator, profile, e2e or CPU baseline)")
    args = ap.parse_args()
    globals()["COUNT"] = args.count
    if args.workload == "large":
        return large_workload(args)
    if args.workload == "serve":
        return serve_workload(args)
    if args.workload == "plain":
        return plain_workload(args)
    if args.workload == "band":
        return band_workload(args)
    if args.workload == "replica":
        return replica_workload(args)
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()

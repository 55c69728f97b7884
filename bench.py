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
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
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
COUNT = 10000  # systems per GPU per step (--count overrides, for small profiling runs)
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


def flops_model(specs, infos_list):
    """Algorithmic work of the dominant class kernels, per step."""
    lu32 = chol32 = lu64 = chol64 = res64 = 0.0
    for (kind, n, r, *_), inf in zip(specs, infos_list):
        route, prec, it = inf["route"], inf["precision"], inf["ir_iters"]
        if route in (6, 5):  # LU
            if prec == 1:
                lu32 += 2.0 / 3.0 * n ** 3
                res64 += 2.0 * n * n * r * (it + 1)
            else:
                lu64 += 2.0 / 3.0 * n ** 3
        elif route == 4:
            if prec == 1:
                chol32 += 1.0 / 3.0 * n ** 3
                res64 += 2.0 * n * n * r * (it + 1)
            else:
                chol64 += 1.0 / 3.0 * n ** 3
    return dict(lu32=lu32, chol32=chol32, lu64=lu64, chol64=chol64, res64=res64)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


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
        X, inf = oracle.solve(A, B)
        return inf
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
        infos = list(ex.map(one, sample))
    dt = time.perf_counter() - t0
    ok = sum(1 for i in infos if i["status"] == 0)
    return {"value": ok / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {len(sample)} of the {len(specs)} systems of the same batch "
                      f"(threads across systems), {dt:.1f} s"}


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
    pk = make_batch(dev, SEED + 7919 * rank, COUNT)
    torch.cuda.synchronize()
    log(f"[rank {rank}] batch generated in {time.perf_counter() - t_gen:.1f}s; "
        f"A bytes {pk['A'].numel() * 8 / 1e9:.2f} GB")
    specs = pk["specs"]
    X = torch.zeros_like(pk["B"])
    infos = torch.zeros(COUNT * asolve.INFO_BYTES, dtype=torch.uint8, device=dev)
    flags = asolve.BERR

    def arm(precision, steps, warmup, profile=False):
        ctx = asolve.Context(precision=precision)
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
    # max over ranks
    tt = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    okt = torch.tensor([float(ok)], dtype=torch.float64, device=dev)
    if dist:
        dist.barrier()
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(okt, op=dist.ReduceOp.SUM)
    total_ms = tt.item()
    value = okt.item() * args.steps / (total_ms / 1e3)
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
                   "precision": "mixed"},
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
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        if dom == "k_scan_batched":
            byt = algorithmic_bytes_scan(specs)
            ach = byt / (per[dom] / 1e3) / 1e9
            result["roofline"] = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                                  "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
                                  "peak_src": peaks["src"]}
        else:
            key32 = "lu32" if dom == "k_lu_class" else "chol32"
            fl = fm[key32]
            ach = fl / (per[dom] / 1e3) / 1e12
            result["roofline"] = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak,
                                  "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": None,
                                  "peak_src": "FP32 FMA: 152 SMs x 128 lanes x 2 flops x 2.07 GHz",
                                  "note": "FP32 factor flops only; the FP64 refinement of the same "
                                          "kernel is not counted"}
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
        return oracle.solve(A, B)[1]

    import concurrent.futures as cf
    t0 = time.perf_counter()
    one(0)
    per = (time.perf_counter() - t0) / max(sub[0][1] ** 3, 1)
    work, m = 0.0, 0
    while m < len(sub) and work < budget * cores / max(per, 1e-15):
        work += sub[m][1] ** 3
        m += 1
    vals = []
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            infos = list(ex.map(one, range(m)))
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                vals.append(sum(1 for i in infos if i["status"] == 0) / dt)
    v = statistics.mean(vals)
    sample = f"first {m} systems of the batched workload per step, threads across systems"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                      "higher_is_better": True, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
                      "steps": args.steps, "warmup": args.warmup, "scaling": "weak",
                      "config": {"workload": WORKLOAD, "systems_per_step": m},
                      "data": "synthetic", "dtype": "f64",
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


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
    ap.add_argument("--quick", action="store_true",
                    help="headline arm only (no FP64 comparator, profile, e2e or CPU baseline)")
    args = ap.parse_args()
    globals()["COUNT"] = args.count
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()

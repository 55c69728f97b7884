"""Autotuner of the batched dense class kernels' panel widths.

For every size bucket (n in [32 i + 1, 32 i + 32]) and each dense kernel
(LU and Cholesky, FP32 factors of the mixed path and FP64 factors of the
plain path), time the batched pipeline on a batch of systems of that size
with each candidate panel width (4, 8, 16, 32; the kernel narrows widths
that do not fit its shared memory) and keep the fastest.  The result is a
JSON table that `asolve.Context(tuning=path)` loads:

    {"device": ..., "nb": {"lu32": [32 widths], "chol32": [...],
                           "lu64": [...], "chol64": [...]}, "ms": {...}}

Usage (on the GPU the table is for):
    python -m paper_2007_11208_gb300.autotune [--out tuning.json] [--buckets 0,4,8,...]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import torch

from . import asolve, build, synth

HERE = os.path.dirname(os.path.abspath(__file__))
CANDIDATES = (4, 8, 16, 32)
KINDS = {"lu32": (0, asolve.PREC_MIXED, "general"), "chol32": (1, asolve.PREC_MIXED, "spd"),
         "lu64": (2, asolve.PREC_FP64, "general"), "chol64": (3, asolve.PREC_FP64, "spd")}


def _batch(n, count, kind, seed, dev):
    specs = [(kind if kind != "general" else "general", n, 1, 1, 1, True)] * count
    pk = synth.packed_batch(specs, seed, device=dev)
    for k in ("n", "nrhs", "a_off", "b_off"):
        pk[k] = pk[k].to(dev)
    return pk


def _time(ctx, pk, count, reps):
    X = torch.zeros_like(pk["B"])
    infos = torch.zeros(count * asolve.INFO_BYTES, dtype=torch.uint8, device=pk["B"].device)
    st = torch.cuda.ExternalStream(ctx.stream)
    for _ in range(2):
        ctx.solve_batched(count, pk["n"], pk["nrhs"], pk["a_off"], pk["b_off"], pk["A"], pk["B"], X, infos,
                          asolve.SYNC)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        rc = ctx.solve_batched(count, pk["n"], pk["nrhs"], pk["a_off"], pk["b_off"], pk["A"], pk["B"], X, infos,
                               asolve.SYNC)
        e1.record(st)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(f"solve_batched: {asolve.strerror(rc)}")
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(buckets=None, per_sm=2, reps=3, kinds=None, seed=77):
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    count = per_sm * sms
    buckets = list(range(16)) if buckets is None else list(buckets)
    kinds = list(KINDS) if kinds is None else list(kinds)
    table = {k: [0] * 32 for k in KINDS}
    times = {}
    for key in kinds:
        kind, prec, mat = KINDS[key]
        ctx = asolve.Context(precision=prec)
        for b in buckets:
            n = 32 * b + 16
            pk = _batch(n, count, mat, seed + b, dev)
            res = {}
            for nb in CANDIDATES:
                if ctx.set_panel_widths(kind, [nb] * 32) != asolve.OK:
                    raise RuntimeError("set_panel_widths")
                res[nb] = _time(ctx, pk, count, reps)
            best = min(res, key=res.get)
            table[key][b] = best
            times[f"{key}:{n}"] = res
            print(f"{key} n={n}: " + ", ".join(f"nb {k}: {v:.2f} ms" for k, v in res.items())
                  + f" -> {best}", flush=True)
            del pk
        ctx.close()
    return {"device": torch.cuda.get_device_name(dev), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
            "systems_per_point": count, "nb": table, "ms": times}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "tuning.json"))
    ap.add_argument("--buckets", default=None,
                    help="comma-separated bucket indices (default 0..15: n <= 512; others keep the built-in rule)")
    ap.add_argument("--kinds", default=None, help="comma-separated subset of lu32,chol32,lu64,chol64")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    buckets = [int(x) for x in args.buckets.split(",")] if args.buckets else None
    kinds = args.kinds.split(",") if args.kinds else None
    res = tune(buckets, reps=args.reps, kinds=kinds)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()

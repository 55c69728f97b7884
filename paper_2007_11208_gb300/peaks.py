"""Measure the arithmetic-pipe peaks of the current GPU and store them.

    python -m paper_2007_11208_gb300.peaks [--out PATH]

Runs the library's issue-rate probes (asolve_pipe_peak: FP32 FMA, FP64 FMA,
FP64 mma.sync m8n8k4), best of five launches each, samples the SM clock
while they run, and writes pipe_peaks.json beside this file.  bench.py takes
the roofline denominators of its FP32-factor / FP64-refinement kernels from
that file.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import time

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "pipe_peaks.json")


def measure(iters: int = 4096, reps: int = 5) -> dict:
    import torch

    from . import asolve, build
    build.build()
    res = {}
    for name, pipe in (("ffma_tflops", asolve.PIPE_FFMA), ("dfma_tflops", asolve.PIPE_DFMA),
                       ("dmma_tflops", asolve.PIPE_DMMA)):
        # about the same duration per launch on each pipe
        it = {asolve.PIPE_FFMA: iters, asolve.PIPE_DFMA: max(1, iters // 16),
              asolve.PIPE_DMMA: max(1, iters // 128)}[pipe]
        best, best_ms = 0.0, 0.0
        for _ in range(reps):
            tf, ms = asolve.pipe_peak(pipe, it)
            if tf > best:
                best, best_ms = tf, ms
        res[name] = best
        res[name.replace("_tflops", "_ms")] = best_ms
    res["gpu_name"] = torch.cuda.get_device_name(0)
    res["sms"] = torch.cuda.get_device_properties(0).multi_processor_count
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--iters", type=int, default=4096)
    a = ap.parse_args()
    q = "clocks.sm,clocks.max.sm"
    smi = None
    try:
        smi = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                "-i", "0", "-lms", "100"], stdout=subprocess.PIPE,
                               stderr=subprocess.DEVNULL, text=True)
    except FileNotFoundError:
        pass
    res = measure(a.iters)
    if smi is not None:
        time.sleep(0.2)
        smi.terminate()
        lines = smi.communicate()[0].strip().splitlines()
        sm = sorted(int(x.split(",")[0]) for x in lines if x.strip())
        mx = [int(x.split(",")[1]) for x in lines if x.strip()]
        if sm:
            res["sm_mhz_median"] = sm[len(sm) // 2]
            res["sm_max_mhz"] = max(mx)
    res["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    res["how"] = ("asolve_pipe_peak: 8 CTAs x 256 threads per SM, 8 independent chains per thread "
                  "(per warp for mma.sync), best of 5 launches, CUDA events")
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()

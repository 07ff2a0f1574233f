"""Measured arithmetic peaks of this GPU for the engine's roofline (gcamps_measure_peaks).

    python -m paper_2511_06672_gb300.peaks [out.json]   # prints them and writes out.json
                                                        # (default profiles/arith_peaks_gb300.json)

FP64 and FP32 fused multiply-add rates and the FP64 tensor-core (m8n8k4) rate, from CUDA-event timings of
long multiply-add chains, with the SM clocks sampled while they run.  bench.py divides the engine's FP64
scoring flops by the FP64 figure of the file (and reports the FP32 work against the FP32 one).
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PEAKS_FILE = os.path.join(ROOT, "profiles", "arith_peaks_gb300.json")


def measure() -> dict:
    from . import _native as N
    lib = N.load()
    out = (C.c_double * 3)()
    rc = lib.gcamps_measure_peaks(out, 3)
    if rc:
        raise RuntimeError(f"gcamps_measure_peaks failed ({rc})")
    return {"fp64_fma_tflops": out[0], "fp32_fma_tflops": out[1], "fp64_mma_tflops": out[2]}


def load(path: str = PEAKS_FILE):
    """The committed measurement, or None."""
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def main():
    from .build import build_library
    build_library()
    smi = None
    try:
        smi = subprocess.Popen(["nvidia-smi", "--query-gpu=name,clocks.sm,clocks.max.sm", "--format=csv,noheader,nounits",
                                "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        pass
    time.sleep(0.3)
    res = measure()
    clocks, name = [], None
    if smi:
        time.sleep(0.2)
        smi.terminate()
        for line in smi.communicate(timeout=5)[0].splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 3:
                name = parts[0]
                try:
                    clocks.append((float(parts[1]), float(parts[2])))
                except ValueError:
                    pass
    res["gpu"] = name
    if clocks:
        sm = sorted(c[0] for c in clocks)
        res["sm_mhz_median"] = sm[len(sm) // 2]
        res["sm_max_mhz"] = max(c[1] for c in clocks)
    res["how"] = ("gcamps_measure_peaks: CUDA events around grids of 8 x SMs blocks x 256 threads, each thread 8 (FP64) "
                  "or 16 (FP32) independent fma chains, or 4 independent m8n8k4 f64 MMA accumulators per warp; "
                  "2 flops per multiply-add; second of two launches timed")
    res["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    print(json.dumps(res))
    path = sys.argv[1] if len(sys.argv) > 1 else PEAKS_FILE
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as fh:
        json.dump(res, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()

"""FP64 and FP32 fused multiply-add rates of this GPU (md_probe_fma_rate), with the
SM clock sampled while the probe runs; JSON on stdout.

    python -m paper_1210_3450_gb300.pipe_rates [--repeats 3]

These are the measured denominators of the FP64 force kernel's roofline (it is
bound by the FP64 pipe); the nominal GB300 FP64 rate (1.25 TFLOP/s) is reported
beside them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NOMINAL_FP64_TFLOPS = 1.25


def measure(repeats: int = 3, iters64: int = 100_000, iters32: int = 5_000_000) -> dict:
    import torch
    from . import build
    from .clocks import ClockSampler
    build.build()
    from . import ljmd
    torch.cuda.set_device(0)
    clk = ClockSampler(0, period_ms=50)
    clk.start()
    r64 = [ljmd.probe_fma_rate(0, iters64) for _ in range(repeats)]
    r32 = [ljmd.probe_fma_rate(1, iters32) for _ in range(repeats)]
    ck = clk.stop()
    d64, d32 = max(r64), max(r32)
    return {"fp64_dfma_per_s": d64, "fp64_tflops": 2 * d64 / 1e12,
            "fp64_fraction_of_nominal": 2 * d64 / 1e12 / NOMINAL_FP64_TFLOPS,
            "fp32_ffma_per_s": d32, "fp32_tflops": 2 * d32 / 1e12,
            "fp32_over_fp64": d32 / d64, "runs": {"fp64": r64, "fp32": r32},
            "iters": {"fp64": iters64, "fp32": iters32}, "clocks": ck}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--repeats", type=int, default=3)
    a = p.parse_args(argv)
    print(json.dumps(measure(a.repeats)))


if __name__ == "__main__":
    main()

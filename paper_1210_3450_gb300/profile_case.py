"""Run a fixed LJ workload through the library for a profiler (ncu) to capture.

    python -m paper_1210_3450_gb300.profile_case --cells 60 --precision fp32 --steps 20

builds an FCC cells^3 x 4 system at rho = 0.8442, T = 0.722 (rc 2.5, skin 0.3,
dt 0.005), sets its state, runs --warmup steps, then --steps steps, and prints
the library's own kernel timing. Inputs are synthetic (lj_inputs).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--cells", type=int, default=60)
    p.add_argument("--rho", type=float, default=0.8442)
    p.add_argument("--temperature", type=float, default=0.722)
    p.add_argument("--rc", type=float, default=2.5)
    p.add_argument("--skin", type=float, default=0.3)
    p.add_argument("--dt", type=float, default=0.005)
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--step-block", type=int, default=None)
    p.add_argument("--step-groups", type=int, default=None)
    p.add_argument("--list-block", type=int, default=None)
    p.add_argument("--step-hint", type=int, default=None)
    p.add_argument("--list-variant", type=int, default=None)
    p.add_argument("--fp64-queue", type=int, default=None)
    p.add_argument("--autotune", action="store_true")
    p.add_argument("--half", action="store_true", help="half pair list with Newton's third law")
    p.add_argument("--observables", action="store_true", help="PE, W, KE, T, P after the steps")
    a = p.parse_args(argv)
    import lj_inputs as li
    from paper_1210_3450_gb300 import build
    build.build()
    from paper_1210_3450_gb300.ljmd import MD_FP32_FORCE, MD_FP64, LJSystem
    n = 4 * a.cells ** 3
    box = li.box_length(n, a.rho)
    x = li.fcc_positions(n, box)
    v = li.maxwell_boltzmann(n, a.temperature, 1000 + a.cells)
    mode = MD_FP32_FORCE if a.precision == "fp32" else MD_FP64
    with LJSystem(box, n, a.rc, a.skin, mode) as s:
        tun = {k: val for k, val in dict(step_block=a.step_block, step_groups=a.step_groups,
                                         list_block=a.list_block, step_hint=a.step_hint,
                                         list_variant=a.list_variant, fp64_queue=a.fp64_queue).items()
               if val is not None}
        if tun:
            s.set_tuning(**tun)
        if a.half:
            from paper_1210_3450_gb300.ljmd import MD_LIST_HALF
            s.set_pair_list(MD_LIST_HALF)
        s.set_state(x, v)
        tuned = None
        if a.autotune:
            from paper_1210_3450_gb300 import autotune
            tuned = autotune.tune(s, a.dt, cache=None, fp32=(mode == MD_FP32_FORCE))
        s.step(a.warmup, a.dt)
        s.set_timing(True)
        s.step(a.steps, a.dt)
        t = s.get_timing()
        listed, inside = s.pair_stats()
        if a.observables:
            t["observables"] = s.observables()
    t.update(n=n, listed_per_particle=listed / n, within_rc_per_particle=inside / n)
    if tuned:
        t["autotune"] = tuned
    print(json.dumps(t))


if __name__ == "__main__":
    main()

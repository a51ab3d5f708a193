"""Autotuner of the kernels' launch shapes.

Times every choice of (step-kernel threads per block, FP32 partner groups per
iteration) and of list-build threads per block on the caller's own system or
batch, with the library's CUDA-event timing, and sets the fastest. Results are
kept in a JSON cache keyed by the workload's shape (precision, particles rounded
to a power of two, density to 0.05, number of systems), so a later run of the
same shape reuses them without timing.

    from paper_1210_3450_gb300 import autotune
    best = autotune.tune(system, dt=0.005)          # LJSystem or LJBatch with a state
"""
from __future__ import annotations

import itertools
import json
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_HERE, "_build", "autotune.json")

STEP_BLOCKS = (64, 128, 256)
STEP_GROUPS = (1, 2)
STEP_HINTS = (0, 1)
LIST_BLOCKS = (64, 128, 256)
LIST_VARIANTS = (0, 1, 2, 3, 4, 5)
FP64_QUEUE = (0, 1)


def shape_key(precision: int, particles: int, density: float, systems: int) -> str:
    return (f"p{precision}-n{2 ** round(math.log2(max(particles, 1)))}-"
            f"rho{round(density * 20) / 20:.2f}-s{systems}")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(system, dt, key: str | None = None, steps: int = 30, cache: str | None = DEFAULT_CACHE,
         fp32: bool = True) -> dict:
    """Time the launch shapes on `system` (it advances by the timed steps) and set
    the fastest. With a cache file and a key already in it, set that instead."""
    if cache and key:
        known = _load(cache).get(key)
        if known:
            system.set_tuning(**known["tuning"])
            return known
    # FP32-force form: partner groups and cache hints; FP64 forms: the queued or
    # plain force loop
    step_choices = list(itertools.product(STEP_BLOCKS, STEP_GROUPS if fp32 else (1,),
                                          STEP_HINTS if fp32 else (0,), (1,) if fp32 else FP64_QUEUE))
    results = {}
    system.step(5, dt)

    def name(c):
        return f"step{c[0]}x{c[1]}h{c[2]}q{c[3]}"

    for c in step_choices:
        system.set_tuning(step_block=c[0], step_groups=c[1], step_hint=c[2], fp64_queue=c[3])
        system.step(2, dt)
        system.set_timing(True)
        system.step(steps, dt)
        t = system.get_timing()
        results[name(c)] = t["step_ms"] / max(t["step_launches"], 1)
    best = min(step_choices, key=lambda c: results[name(c)])
    system.set_tuning(step_block=best[0], step_groups=best[1], step_hint=best[2], fp64_queue=best[3])
    list_times = {}
    for lb, lv in itertools.product(LIST_BLOCKS, LIST_VARIANTS):
        system.set_tuning(list_block=lb, list_variant=lv)
        system.set_timing(True)
        system.build_list() if hasattr(system, "build_list") else None
        system.step(steps, dt)
        t = system.get_timing()
        if t["list_launches"]:
            list_times[(lb, lv)] = t["list_ms"] / t["list_launches"]
    lbest, lvar = min(list_times, key=list_times.get) if list_times else (128, 0)
    system.set_tuning(list_block=lbest, list_variant=lvar)
    system.set_timing(False)
    out = dict(tuning=system.get_tuning(),
               step_ms=results, list_ms={f"{k[0]}v{k[1]}": v for k, v in list_times.items()})
    if cache and key:
        data = _load(cache)
        data[key] = out
        _save(cache, data)
    return out

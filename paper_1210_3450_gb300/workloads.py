"""Runners for the multi-system and long workloads (JSON results on stdout).

    python -m paper_1210_3450_gb300.workloads batched     [--count 256 --steps 2000]
    python -m paper_1210_3450_gb300.workloads cavitation  [--cells 160 --steps 20000]
    python -m paper_1210_3450_gb300.workloads serve       [--rate 200 --duration 60]
    python -m paper_1210_3450_gb300.workloads serve-scaled [--load 0.8 --duration 60]

* batched: independent replica systems (N log-uniform in [500, 32000], rho in
  [0.60, 0.85], T in [0.7, 1.2], rc 2.5, dt 0.005) stepped together, one launch
  per kernel per step for the whole batch.
* cavitation: a 16,384,000-particle liquid at rho 0.70 held at T = 0.90 by a
  Nose-Hoover thermostat (Sec. 4.1; or velocity rescaling every 10 steps with
  --thermostat rescale), then expanded uniformly by 1.05 per axis
  (x -> 1.05 x, L -> 1.05 L, momenta kept; Sec. 4.1 of the paper uses 1.025) and
  run NVE with rc = 3.0 (the two-phase region: bubbles nucleate); reports
  particle-steps/s, list rebuilds, and every 1000 steps the pressure and the
  bubbles found as in Sec. 4.2 (subcells of side 3, gas below density 0.2).
* serve / serve-scaled: Poisson arrivals of LJ runs (N log-uniform in
  [1e3, 1e6], rho in [0.6, 0.85], T in [0.722, 1.2], steps in [1e3, 1e4])
  through the continuous-batching server; serve-scaled sets the arrival rate to
  a fraction of the measured capacity.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _cuda_time(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def batched(count=256, steps=2000, warmup=20, precision=1, seed=1004, tune=True,
            tune_cache: str | None = None) -> dict:
    """The replica batch; with tune=True the autotuner picks the launch shapes on
    the batch itself first (or takes them from its keyed cache) and the chosen
    tuning is part of the result."""
    import torch
    import lj_inputs as li
    from . import autotune, ljmd
    syss = li.batch_systems(count=count, seed=seed)
    n_tot = sum(c.n for c in syss)
    b = ljmd.LJBatch(systems=[(c.n, c.box, c.rc, c.skin) for c in syss], precision=precision)
    for k, c in enumerate(syss):
        b.set_state(k, c.x, c.v)
    dts = [c.dt for c in syss]
    stream = torch.cuda.Stream()
    tuned = None
    if tune:
        key = autotune.shape_key(precision, n_tot, sum(c.rho * c.n for c in syss) / n_tot, count)
        tuned = autotune.tune(b, dts, key=key, cache=tune_cache or autotune.DEFAULT_CACHE,
                              fp32=(precision == 1))
        tuned = dict(key=key, tuning=tuned["tuning"])
    b.step_async(warmup, dts, stream)
    # per-kernel times: a host-driven pass with CUDA events around each launch
    b.set_timing(True)
    b.step_async(max(min(steps // 4, 200), 20), dts, stream)
    torch.cuda.synchronize()
    tm = b.get_timing()
    b.set_timing(False)
    r0 = sum(b.stats(k)["rebuilds"] for k in range(count))
    # the timed region: graph-captured chunks (the library's default stepping)
    sec = _cuda_time(lambda: b.step_async(steps, dts, stream), stream)
    launches = b.get_timing()["launches"]
    small = sum(1 for c in syss if math.floor(c.box / (c.rc + c.skin)) < 3)
    rebuilds = sum(b.stats(k)["rebuilds"] for k in range(count)) - r0
    b.close()
    return dict(workload=f"{count} replicas, N log-uniform [500, 32000], total N={n_tot}",
                systems=count, particles=n_tot, steps=steps, seconds=sec,
                value=n_tot * steps / sec, unit="particle-steps/s", ms_per_step=sec * 1e3 / steps,
                all_pairs_systems=small, list_builds=rebuilds,
                kernel_ms_per_step=tm["step_ms"] / max(tm["step_launches"], 1),
                list_build_ms_per_launch=tm["list_ms"] / max(tm["list_launches"], 1),
                launches_per_step=launches / steps, autotuned=tuned,
                precision="fp32-force" if precision == 1 else "fp64")


def cavitation(cells=160, equil_steps=2000, rescale_every=10, steps=20000, alpha=1.05, precision=1,
               obs_every=1000, thermostat="nose-hoover", tau=0.5) -> dict:
    import numpy as np
    import torch
    import lj_inputs as li
    from . import ljmd
    cfg = li.config_cavitation(cells)
    n = cfg.n
    s = ljmd.LJSystem(cfg.box, n, cfg.rc, cfg.skin, precision)
    s.set_state(cfg.x, cfg.v)
    t_eq = time.perf_counter()
    if thermostat == "nose-hoover":
        # Nose-Hoover with thermostat period tau: Q = g T tau^2 / (4 pi^2) ~ g T tau^2 / 40
        q = 3.0 * (n - 1) * cfg.temperature * tau * tau / (4.0 * math.pi ** 2)
        zeta, eta = s.step_nvt(equil_steps, cfg.dt, cfg.temperature, q)
    else:
        for _ in range(equil_steps // rescale_every):
            s.step(rescale_every, cfg.dt)
            t = 2.0 * s.kinetic_energy() / (3.0 * (n - 1))
            s.scale_velocities(math.sqrt(cfg.temperature / t))
    t_eq = time.perf_counter() - t_eq
    obs0 = s.observables()
    xd = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    vd = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    s.get_state_dev(xd, vd)
    torch.cuda.synchronize()
    s.close()
    # uniform adiabatic expansion: lengths scaled, momenta kept (Sec. 4.1)
    xd *= alpha
    box = cfg.box * alpha
    s = ljmd.LJSystem(box, n, cfg.rc, cfg.skin, precision)
    s.set_state_dev(xd, vd)
    torch.cuda.synchronize()
    del xd, vd
    stream = torch.cuda.Stream()
    s.step_async(1, cfg.dt, stream)
    torch.cuda.synchronize()
    # per-kernel times from a short host-driven pass; the timed run below steps in
    # graph-captured chunks
    s.set_timing(True)
    s.step_async(50, cfg.dt, stream)
    torch.cuda.synchronize()
    tm = s.get_timing()
    s.set_timing(False)
    r0 = s.stats()["rebuilds"]
    sec = 0.0
    series = []
    done = 0
    while done < steps:
        k = min(obs_every, steps - done)
        sec += _cuda_time(lambda: s.step_async(k, cfg.dt, stream), stream)
        done += k
        o = s.observables()
        b = s.bubbles(3.0, 0.2)
        series.append(dict(step=done, pressure=o["pressure"], temperature=o["temperature"],
                           pe_per_particle=o["pe"] / n, bubbles=b["n_bubbles"],
                           largest_bubble_subcells=int(b["sizes"][0]) if b["n_bubbles"] else 0,
                           gas_subcells=int(b["sizes"].sum())))
    rebuilds = s.stats()["rebuilds"] - r0
    s.close()
    return dict(workload=f"cavitation N={n}, rho 0.70 -> {0.70 / alpha ** 3:.4f}, T 0.90, rc 3.0",
                particles=n, steps=steps, seconds=sec, value=n * steps / sec, unit="particle-steps/s",
                ms_per_step=sec * 1e3 / steps, list_builds=rebuilds,
                steps_per_build=steps / max(rebuilds, 1),
                kernel_ms_per_step=tm["step_ms"] / max(tm["step_launches"], 1),
                list_build_ms_per_launch=tm["list_ms"] / max(tm["list_launches"], 1),
                equilibration=dict(steps=equil_steps, thermostat=thermostat, seconds=t_eq,
                                   pressure=obs0["pressure"], temperature=obs0["temperature"]),
                series=series, precision="fp32-force" if precision == 1 else "fp64")


def mean_request_work() -> float:
    """E[N] E[steps] of the served workload: N log-uniform on [1e3, 1e6],
    steps uniform on [1e3, 1e4]."""
    a, b = 1e3, 1e6
    en = (b - a) / math.log(b / a)
    return en * 5500.0


def serve_run(rate, duration, budget_gb=100.0, chunk=100, drain_limit=None, precision=1,
              policy="shared") -> dict:
    from . import ljmd, serve
    reqs = serve.requests_from_workload(rate, duration)
    srv = serve.MDServer(int(budget_gb * 1e9), precision, chunk=chunk, policy=policy)
    try:
        out = srv.run(reqs, drain_limit=drain_limit)
    finally:
        srv.close()
    out.update(rate=rate, duration=duration, budget_gb=budget_gb, chunk=chunk, policy=policy,
               offered_particle_steps_per_s=rate * mean_request_work())
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("which", choices=["batched", "cavitation", "serve", "serve-scaled"])
    p.add_argument("--count", type=int, default=256)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--cells", type=int, default=160)
    p.add_argument("--equil-steps", type=int, default=2000)
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--duration", type=float, default=60.0)
    p.add_argument("--load", type=float, default=0.8)
    p.add_argument("--capacity", type=float, default=None, help="particle-steps/s (else measured)")
    p.add_argument("--budget-gb", type=float, default=100.0)
    p.add_argument("--drain-limit", type=float, default=None)
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    p.add_argument("--thermostat", choices=["nose-hoover", "rescale"], default="nose-hoover")
    p.add_argument("--no-tune", action="store_true", help="batched: default launch shapes, no autotuning")
    a = p.parse_args(argv)
    from . import build
    build.build()
    prec = 1 if a.precision == "fp32" else 0
    if a.which == "batched":
        out = batched(a.count, a.steps or 2000, precision=prec, tune=not a.no_tune)
    elif a.which == "cavitation":
        out = cavitation(a.cells, a.equil_steps, steps=a.steps or 20000, precision=prec,
                         thermostat=a.thermostat)
    elif a.which == "serve":
        out = serve_run(a.rate, a.duration, a.budget_gb, drain_limit=a.drain_limit, precision=prec)
    else:
        cap = a.capacity or batched(64, 200, precision=prec)["value"]
        rate = a.load * cap / mean_request_work()
        out = serve_run(rate, a.duration, a.budget_gb, drain_limit=a.drain_limit, precision=prec)
        out.update(capacity_particle_steps_per_s=cap, load=a.load)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

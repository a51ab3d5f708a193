#!/usr/bin/env python
"""Benchmark of the GB300 truncated-LJ MD hot path (one JSON line on stdout).

Workload: the 2,048,000-particle LJ fluid (FCC 80^3 x 4, rho = 0.8442, T = 0.722,
rc = 2.5, skin 0.3, dt = 0.005), synthetic and seeded. One bench "step" is one
velocity-Verlet step of the whole hot path: force over the pair list, kicks,
drift, list-validity check and, when it triggers, the cell binning, sort and
list rebuild. Observables are not computed inside the timed region.

`value` is particle-steps/s (the paper's MUPS x 1e6, Sec. 3.2) of the FP32-force
form (pair forces in FP32, integration / lists / energies in FP64); the plain
FP64 form is measured on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the plain FP64 CPU oracle on this machine's host cores
on a bounded sample of the same workload. With N > 1 (torchrun) every rank runs
an independent replica ("replicas only": the path has no data exchange between
GPUs here); value = particle-steps of all ranks / max elapsed time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (FP32-force vs FP64) + roofline %; p50/p99 batched MD latency"
UNIT = "particle-steps/s"
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 (vector and tensor), recipe table

# Compulsory bytes per particle-step of the fused FP32 force + integration kernel
# (k_step_fp32), by name; the list adds 4 bytes per listed partner.
FP32_STEP_BYTES = {
    "partner_shadows_once": 16,   # every particle's 16-byte shadow is gathered at least once
    "position_read": 32,          # own FP64 position (double4)
    "position_write": 32,         # drifted position into the other buffer
    "velocity_read": 32,
    "velocity_write": 32,
    "shadow_write": 16,           # fixed-point shadow of the drifted position
    "reference_shadow_read": 16,  # shadow at the last list build (validity check)
    "list_length": 4,
}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--skip-cpu-baseline", action="store_true")
    p.add_argument("--skip-batched", action="store_true", help="no batched-replica / serving sub-results")
    p.add_argument("--skip-cavitation", action="store_true", help="no cavitation-run sub-result")
    p.add_argument("--skip-serve-spec", action="store_true",
                   help="no as-specified serving run (200 requests/s for 60 s)")
    p.add_argument("--serve-seconds", type=float, default=20.0)
    p.add_argument("--cavitation-steps", type=int, default=2000)
    return p.parse_args()


def workload_config():
    import lj_inputs as li
    cfg = li.config_large_fluid()
    desc = {
        "workload": f"{cfg.name}: N={cfg.n} (FCC 80^3 x 4), rho={cfg.rho}, T={cfg.temperature}, "
                    f"rc={cfg.rc}, skin={cfg.skin}, dt={cfg.dt}, velocity Verlet",
        "particles": cfg.n,
        "box": cfg.box,
        "l2": "inputs larger than L2 (pair list ~0.7 GB, state ~0.4 GB per form)",
        "parallelism": "replicas",
    }
    return cfg, desc


# ------------------------------------------------------------------ helpers

# the device code of the profiled kernels (host code cannot change their traffic)
KERNEL_SOURCES = ("ljmd_kernels.cu", "ljmd_dev.cuh", "ljmd_math.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1210_3450_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("kernel_sources") != kernel_source_hash():
        return None
    return e["dram_bytes_per_particle_step"] * n


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ our arm

def time_form(ljmd, cfg, precision, steps, warmup, stream, clocks, dist):
    """Two passes over the same run: a host-driven pass with CUDA events around
    every kernel launch (per-kernel durations for the roofline), then the timed
    region proper, stepped as the library steps by default (graph-captured
    chunks, the host reading the control words once per chunk)."""
    import torch
    s = ljmd.LJSystem(cfg.box, cfg.n, cfg.rc, cfg.skin, precision)
    s.set_state(cfg.x, cfg.v)
    s.step_async(warmup, cfg.dt, stream)
    torch.cuda.synchronize()
    s.set_timing(True)
    s.step_async(max(min(steps, 200), 20), cfg.dt, stream)
    torch.cuda.synchronize()
    tm = s.get_timing()
    s.set_timing(False)
    r0 = s.stats()["rebuilds"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark(True)
    e0.record(stream)
    s.step_async(steps, cfg.dt, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = s.get_timing()["launches"]
    st = s.stats()
    listed, inside = s.pair_stats()
    s.close()
    return dict(ms=ms, timing=tm, listed=listed, inside=inside, rebuilds=st["rebuilds"] - r0, stats=st,
                launches=launches)


def e2e_run(ljmd, cfg, precision, steps):
    """Public-API run with host buffers in pinned memory: set_state (H2D), steps,
    get_state and observables (D2H), all inside the timed region."""
    import torch

    def pinned():
        return torch.empty((cfg.n, 3), dtype=torch.float64, pin_memory=True).numpy()

    xin, vin, xout, vout = pinned(), pinned(), pinned(), pinned()
    xin[:] = cfg.x
    vin[:] = cfg.v
    s = ljmd.LJSystem(cfg.box, cfg.n, cfg.rc, cfg.skin, precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(xin, vin)
    s.step(steps, cfg.dt)
    s.get_state(out=(xout, vout))
    o = s.observables()
    t1 = time.perf_counter()
    s.close()
    return dict(seconds=t1 - t0, h2d=2 * 8 * 3 * cfg.n, d2h=2 * 8 * 3 * cfg.n + 5 * 8, obs=o)


_SAMPLE_M = 24  # the oracle's bounded sample: an FCC 24^3 x 4 block (55,296 particles)


def _oracle_sample_rate(args):
    """Particle-steps/s of the oracle on the bounded sample (run in one process):
    per-step time = (t(1 + k steps) - t(1 step)) / k, so the list build at the
    start of each run is excluded once."""
    rho, temperature, rc, skin, dt, k = args
    import lj_inputs as li
    import oracle
    n = 4 * _SAMPLE_M ** 3
    box = li.box_length(n, rho)
    x = li.fcc_positions(n, box)
    v = li.maxwell_boltzmann(n, temperature, 1002)
    t = time.perf_counter()
    oracle.run(x, v, box, rc, skin, 1, dt)
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.run(x, v, box, rc, skin, 1 + k, dt)
    tk = time.perf_counter() - t
    return n * k / max(tk - t1, 1e-9), tk + t1


def cpu_baseline(cfg, budget_s=15.0):
    """The oracle as it stands on a bounded sample of the workload (an FCC 24^3 x 4
    block at the same density, temperature, cutoff, skin and dt): one thread, and
    all host cores as independent oracle processes on the same sample (the oracle
    is single-threaded; started with spawn, its results are the same per process)."""
    import multiprocessing as mp
    n = 4 * _SAMPLE_M ** 3
    rate1, _ = _oracle_sample_rate((cfg.rho, cfg.temperature, cfg.rc, cfg.skin, cfg.dt, 2))
    k = int(max(2, min(40, budget_s * rate1 / n)))
    rate1, _ = _oracle_sample_rate((cfg.rho, cfg.temperature, cfg.rc, cfg.skin, cfg.dt, k))
    cores = os.cpu_count() or 1
    sample = (f"FCC {_SAMPLE_M}^3x4 = {n} particles at rho={cfg.rho}, T={cfg.temperature}, "
              f"rc={cfg.rc}, skin={cfg.skin}, dt={cfg.dt}; {k} steps timed (initial list build "
              f"excluded)")
    out = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample + "; single thread"}
    kall = max(2, k // 2)
    try:
        ctx = mp.get_context("spawn")
        t = time.perf_counter()
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_sample_rate, [(cfg.rho, cfg.temperature, cfg.rc, cfg.skin, cfg.dt, kall)] * cores)
        wall = time.perf_counter() - t
        # whole-job throughput: particle-steps of all processes over the slowest one's
        # timed steps (the per-process rates are summed over a shared wall window)
        out["all_cores"] = {"value": sum(r[0] for r in res), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample.replace(f"{k} steps", f"{kall} steps")
                                      + f"; {cores} independent single-thread oracle processes at once",
                            "wall_s": round(wall, 2)}
    except Exception as e:  # the single-thread figure stands on its own
        out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return out


def replica_totals(dist, seconds: float, units: float, device: str = "cpu") -> tuple[float, float]:
    """Whole-job figures of independent replicas: the slowest rank's time (max over
    ranks) and the units every rank processed (sum over ranks). Without a process
    group, this rank's own figures."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cavitation_leg(steps: int) -> dict:
    """The cavitation-shaped run (16,384,000 particles at rho 0.70, T 0.90, rc 3.0):
    Nose-Hoover equilibration, uniform expansion by 1.05 per axis, then `steps` NVE
    steps in graph-captured chunks (timed), with pressure and bubbles at the end."""
    from paper_1210_3450_gb300 import workloads
    r = workloads.cavitation(cells=160, equil_steps=2000, steps=steps, obs_every=steps)
    last = r["series"][-1]
    return {"workload": r["workload"], "value": round(r["value"], 1), "unit": r["unit"],
            "ms_per_step": round(r["ms_per_step"], 4), "steps": r["steps"], "list_builds": r["list_builds"],
            "steps_per_build": round(r["steps_per_build"], 2),
            "kernel_ms_per_step": round(r["kernel_ms_per_step"], 4),
            "list_build_ms": round(r["list_build_ms_per_launch"], 4),
            "equilibration": {k: (round(v, 5) if isinstance(v, float) else v)
                              for k, v in r["equilibration"].items()},
            "final": {"pressure": round(last["pressure"], 6), "temperature": round(last["temperature"], 6),
                      "bubbles": last["bubbles"], "largest_bubble_subcells": last["largest_bubble_subcells"],
                      "gas_subcells": last["gas_subcells"]},
            "note": "NVE phase timed with CUDA events; observables and bubbles outside the timed chunks"}


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1210_3450_gb300.ljmd as ljmd
    from paper_1210_3450_gb300.clocks import ClockSampler
    cfg, desc = workload_config()
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local)
    clocks.start()
    r32 = time_form(ljmd, cfg, ljmd.MD_FP32_FORCE, args.steps, args.warmup, stream, clocks, dist)
    r64_steps = max(args.steps // 10, 100)
    r64 = time_form(ljmd, cfg, ljmd.MD_FP64, r64_steps, max(args.warmup // 4, 3), stream, clocks, dist)
    ck = clocks.stop()

    sec32, units32 = replica_totals(dist, r32["ms"] / 1e3, float(cfg.n * args.steps), "cuda")
    sec64, units64 = replica_totals(dist, r64["ms"] / 1e3, float(cfg.n * r64_steps), "cuda")
    ms32, ms64 = sec32 * 1e3, sec64 * 1e3
    value = units32 / sec32
    value64 = units64 / sec64

    e2e = e2e_run(ljmd, cfg, ljmd.MD_FP32_FORCE, args.steps)
    e2e_sec, e2e_units = replica_totals(dist, e2e["seconds"], float(cfg.n * args.steps), "cuda")
    e2e_val = e2e_units / e2e_sec

    # the other workloads and the baselines: one GPU only (under torchrun every rank
    # runs the headline replica alone)
    extras = world == 1 and rank == 0
    batched = serve = serve_spec = cav = rates = None
    if extras:
        rates = {"fp64_dfma_per_s": ljmd.probe_fma_rate(0, 100_000),
                 "fp32_ffma_per_s": ljmd.probe_fma_rate(1, 5_000_000)}
    if extras and not args.skip_batched:
        from paper_1210_3450_gb300 import workloads
        batched = workloads.batched(count=256, steps=1000, warmup=10)
        rate = 0.8 * batched["value"] / workloads.mean_request_work()
        serve = workloads.serve_run(rate, args.serve_seconds, budget_gb=100.0)
        if not args.skip_serve_spec:
            serve_spec = workloads.serve_run(200.0, 60.0, budget_gb=100.0, drain_limit=60.0)
    if extras and not args.skip_cavitation:
        cav = cavitation_leg(args.cavitation_steps)

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    hbm_peak, peak_src = load_peaks()
    n = cfg.n
    # fused FP32 step kernel: compulsory bytes per particle-step, by name
    lp = r32["listed"] / n
    breakdown = {"list_words": round(4.0 * lp, 1), **FP32_STEP_BYTES}
    bytes_pp = sum(breakdown.values())
    t32 = r32["timing"]
    k_ms = t32["step_ms"] / max(t32["step_launches"], 1)
    achieved = bytes_pp * n / (k_ms / 1e3) / 1e9
    traffic = profiled_traffic("k_step_fp32", n)
    roof = {"bound": "hbm", "kernel": "k_step_fp32 (fused FP32 pair force + velocity Verlet)",
            "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
            "algorithmic_bytes_per_particle_step": round(bytes_pp, 1), "bytes_breakdown": breakdown,
            "achieved_dram": round(traffic / (k_ms / 1e3) / 1e9, 1) if traffic else None,
            "frac_dram": round(traffic / (k_ms / 1e3) / 1e9 / hbm_peak, 4) if traffic else None,
            "avg_launch_ms": round(k_ms, 4),
            "avg_launch_ms_source": "CUDA events around each launch (host-driven pass of the same run)"}
    # FP64 step kernel: FP64-pipe bound; flops as the method needs them: the
    # separation and r^2 of every listed pair (10, an FMA counted as 2) and the
    # force of every pair inside rc (16)
    t64 = r64["timing"]
    k64 = t64["step_ms"] / max(t64["step_launches"], 1)
    lp64 = r64["listed"] / n
    in64 = r64["inside"] / n
    flops_pp = 10.0 * lp64 + 16.0 * in64
    ach64 = flops_pp * n / (k64 / 1e3) / 1e12
    roof64 = {"bound": "alu", "kernel": "k_step_fp64 (classified, queued FP64 pair force + velocity Verlet)",
              "achieved": round(ach64, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
              "frac": round(ach64 / FP64_PEAK_TFLOPS, 4),
              "traffic": profiled_traffic("k_step_fp64", n),
              "peak_source": "nominal GB300 FP64 (1.25 TFLOP/s, recipe table)",
              "algorithmic_flops_per_particle_step": round(flops_pp, 1),
              "flop_count": "10 per listed pair (separation, r^2) + 16 per pair inside rc (force, accumulation)",
              "avg_launch_ms": round(k64, 4)}
    if rates:
        meas = 2.0 * rates["fp64_dfma_per_s"] / 1e12
        roof64.update(peak_measured=round(meas, 4), frac_measured=round(ach64 / meas, 4),
                      peak_measured_source="md_probe_fma_rate: DFMA chains on every SM, this run")
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms32 / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "dtype_detail": "pair forces f32; positions, velocities, list tests, energies f64",
        "data": "synthetic", "config": desc,
        "fp64": {"value": round(value64, 1), "unit": UNIT, "steps": r64_steps,
                 "ms_per_step": round(ms64 / r64_steps, 5), "dtype": "f64", "roofline": roof64,
                 "rebuilds": r64["rebuilds"]},
        "fp32_speedup_over_fp64": round(value / value64, 3),
        "roofline": roof,
        "rebuilds": r32["rebuilds"],
        "pairs_per_particle": {"listed": round(lp, 3), "within_rc": round(r32["inside"] / n, 3)},
        "kernel_ms_per_step": {"step": round(k_ms, 4),
                               "list_build_per_rebuild": round(t32["list_ms"] / max(t32["list_launches"], 1), 4),
                               "binning_per_rebuild": round(t32["bin_ms"] / max(t32["rebuilds"], 1), 4)},
        "gpu_launches": int(r32["launches"]),
        "e2e": {"value": round(e2e_val, 1), "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d"] // args.steps, "d2h_bytes_per_step": e2e["d2h"] // args.steps,
                "note": ("set_state (x, v from pinned host memory) + steps + get_state (into pinned host "
                         "memory) + observables through the C ABI, wall clock")},
        "clocks": ck,
    }
    if rates:
        line["pipe_rates"] = {"fp64_tflops": round(2.0 * rates["fp64_dfma_per_s"] / 1e12, 4),
                              "fp32_tflops": round(2.0 * rates["fp32_ffma_per_s"] / 1e12, 2),
                              "source": "md_probe_fma_rate (FMA = 2 flops), this run"}
    if batched:
        line["batched"] = {k: batched[k] for k in ("workload", "value", "unit", "ms_per_step", "steps",
                                                    "list_builds", "launches_per_step", "autotuned")}
    if serve:
        line["serve"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in serve.items()}
        line["serve"]["note"] = ("Poisson arrivals at 80% of the batched capacity, N log-uniform "
                                 "[1e3, 1e6], steps [1e3, 1e4]; latency includes queueing")
    if serve_spec:
        line["serve_as_specified"] = {k: (round(v, 4) if isinstance(v, float) else v)
                                      for k, v in serve_spec.items()}
        line["serve_as_specified"]["note"] = (
            "Poisson arrivals at 200 requests/s for 60 s (offered load about 40x one GPU); the run stops "
            "60 s after the last arrival; latency percentiles over the completed requests, unfinished "
            "ones counted and their remaining work projected at the measured rate")
    if cav:
        line["cavitation"] = cav
    if not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import lj_inputs as li
    import oracle
    cfg, desc = workload_config()
    # bounded sample: an FCC block small enough that W + K oracle steps take ~2 min
    probe_m = 12
    pn = 4 * probe_m ** 3
    pbox = li.box_length(pn, cfg.rho)
    px = li.fcc_positions(pn, pbox)
    pv = li.maxwell_boltzmann(pn, cfg.temperature, 1002)
    t = time.perf_counter()
    oracle.run(px, pv, pbox, cfg.rc, cfg.skin, 4, cfg.dt)
    rate = pn * 4 / (time.perf_counter() - t)
    total = max(args.steps + args.warmup, 1)
    m = int(round((120.0 * rate / total / 4) ** (1 / 3)))
    m = max(6, min(m, 80))
    n = 4 * m ** 3
    box = li.box_length(n, cfg.rho)
    x = li.fcc_positions(n, box)
    v = li.maxwell_boltzmann(n, cfg.temperature, 1002)
    w = oracle.run(x, v, box, cfg.rc, cfg.skin, max(args.warmup, 1), cfg.dt)
    t = time.perf_counter()
    oracle.run(w["x"], w["v"], box, cfg.rc, cfg.skin, args.steps, cfg.dt)
    sec = time.perf_counter() - t
    value = n * args.steps / sec
    sample = (f"FCC {m}^3x4 = {n} particles at rho={cfg.rho}, T={cfg.temperature}, rc={cfg.rc}, "
              f"skin={cfg.skin}, dt={cfg.dt}; {args.steps} timed steps after {args.warmup}; single thread")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": desc,
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

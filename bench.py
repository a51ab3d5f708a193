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
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (FP32-force vs FP64) + roofline %; p50/p99 batched MD latency"
UNIT = "particle-steps/s"
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 (vector and tensor), recipe table


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--skip-cpu-baseline", action="store_true")
    p.add_argument("--skip-batched", action="store_true", help="no batched-replica / serving sub-results")
    p.add_argument("--serve-seconds", type=float, default=20.0)
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


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed regions."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None
        self.windows = []

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, begin: bool):
        t = time.time()
        if begin:
            self.windows.append([t, None])
        else:
            self.windows[-1][1] = t

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [q.strip() for q in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(rows), "reasons": reasons}


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


def cpu_baseline(cfg, budget_s=20.0):
    """The oracle (single thread, as it stands) on a bounded sample of the workload:
    an FCC m^3 x 4 block at the same density, temperature, cutoff, skin and dt;
    per-step time = (t(run of 1 + k steps) - t(run of 1 step)) / k, so the list
    build at the start of each run is excluded once."""
    import lj_inputs as li
    import oracle
    m = 24
    n = 4 * m ** 3
    box = li.box_length(n, cfg.rho)
    x = li.fcc_positions(n, box)
    v = li.maxwell_boltzmann(n, cfg.temperature, 1002)
    t = time.perf_counter()
    oracle.run(x, v, box, cfg.rc, cfg.skin, 1, cfg.dt)
    t1 = time.perf_counter() - t
    k = max(2, int(budget_s / max(t1, 1e-3)))
    k = min(k, 40)
    t = time.perf_counter()
    oracle.run(x, v, box, cfg.rc, cfg.skin, 1 + k, cfg.dt)
    tk = time.perf_counter() - t
    per_step = max((tk - t1) / k, 1e-9)
    return {"value": n / per_step, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FCC {m}^3x4 = {n} particles at rho={cfg.rho}, T={cfg.temperature}, "
                      f"rc={cfg.rc}, skin={cfg.skin}, dt={cfg.dt}; {k} steps timed "
                      f"(initial list build excluded); single thread"}


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
    cfg, desc = workload_config()
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local)
    clocks.start()
    r32 = time_form(ljmd, cfg, ljmd.MD_FP32_FORCE, args.steps, args.warmup, stream, clocks, dist)
    r64_steps = max(args.steps // 4, 10)
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

    batched = serve = None
    if not args.skip_batched and rank == 0:
        from paper_1210_3450_gb300 import workloads
        batched = workloads.batched(count=256, steps=500, warmup=10)
        rate = 0.8 * batched["value"] / workloads.mean_request_work()
        serve = workloads.serve_run(rate, args.serve_seconds, budget_gb=100.0)

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    hbm_peak, peak_src = load_peaks()
    n = cfg.n
    # fused FP32 step kernel: algorithmic bytes per particle-step
    lp = r32["listed"] / n
    bytes_pp = 4.0 * lp + 208.0
    t32 = r32["timing"]
    k_ms = t32["step_ms"] / max(t32["step_launches"], 1)
    achieved = bytes_pp * n / (k_ms / 1e3) / 1e9
    traffic = profiled_traffic("k_step_fp32", n)
    roof = {"bound": "hbm", "kernel": "k_step<fp32> (fused force + velocity Verlet)",
            "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
            "algorithmic_bytes_per_particle_step": round(bytes_pp, 1),
            "avg_launch_ms": round(k_ms, 4),
            "avg_launch_ms_source": "CUDA events around each launch (host-driven pass of the same run)"}
    # FP64 step kernel: FP64-pipe bound (FMA = 2 flops)
    t64 = r64["timing"]
    k64 = t64["step_ms"] / max(t64["step_launches"], 1)
    lp64 = r64["listed"] / n
    in64 = r64["inside"] / n
    flops_pp = 8.0 * lp64 + 19.0 * in64 + 26.0
    ach64 = flops_pp * n / (k64 / 1e3) / 1e12
    roof64 = {"bound": "alu", "kernel": "k_step<fp64>", "achieved": round(ach64, 4),
              "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(ach64 / FP64_PEAK_TFLOPS, 4),
              "traffic": profiled_traffic("k_step_fp64", n),
              "peak_source": "nominal GB300 FP64 (1.25 TFLOP/s); probe-measured DFMA rate 1.05 TFLOP/s",
              "algorithmic_flops_per_particle_step": round(flops_pp, 1), "avg_launch_ms": round(k64, 4)}
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
    if batched:
        line["batched"] = {k: batched[k] for k in ("workload", "value", "unit", "ms_per_step", "steps",
                                                    "list_builds", "launches_per_step")}
    if serve:
        line["serve"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in serve.items()}
        line["serve"]["note"] = ("Poisson arrivals at 80% of the batched capacity, N log-uniform "
                                 "[1e3, 1e6], steps [1e3, 1e4]; latency includes queueing")
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

"""Continuous-batching server for LJ MD runs on one GPU.

Requests (N, density, temperature, number of steps) arrive over time. Each is
admitted into a device-resident arena (``LJBatch``) as soon as its particles,
cells and pair list fit in the arena's free space, whose total size is fixed by
an HBM budget; all admitted runs then advance together, one launch per kernel
per step for the whole mix, in chunks of steps. A run that has done its steps
is read back (final state and observables) and its arena space is freed for
the next request. Requests that arrive while others run join at the next chunk
boundary; a run's result does not depend on the other runs in the mix.

    python -m paper_1210_3450_gb300.serve --rate 200 --duration 60 --budget-gb 100

prints a JSON summary (p50 / p99 latency including queueing, throughput).
"""
from __future__ import annotations

import argparse
import collections
import concurrent.futures as cf
import json
import math
import os
import sys
import time
from dataclasses import dataclass, field

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from . import ljmd  # noqa: E402

# Device bytes per particle slot of the arena (positions x2, velocity, two
# reference copies, forces, half-list force sums, shadow positions x2, float
# positions for the list build, indices and rebuild scratch).
SLOT_BYTES = 324
LIST_WORD_BYTES = 4
CELL_BYTES = 8


def arena_for_budget(budget_bytes: int, max_systems: int = 4096, list_share: float = 0.62) -> dict:
    """Arena capacities that fit in budget_bytes of device memory."""
    list_words = int(budget_bytes * list_share / LIST_WORD_BYTES)
    rest = budget_bytes - list_words * LIST_WORD_BYTES
    slots = int(rest * 0.95 / SLOT_BYTES)
    cells = int(rest * 0.05 / CELL_BYTES)
    return dict(slots=slots, cells=cells, list_words=list_words, max_systems=max_systems)


@dataclass(eq=False)
class Request:
    id: int
    arrival: float
    n: int
    rho: float
    temperature: float
    steps: int
    seed: int
    rc: float = 2.5
    skin: float = 0.3
    dt: float = 0.005
    cancel_after: float = math.nan  # seconds after arrival at which the client cancels
    # initial state: "fcc" fills the box with an FCC lattice; "droplet" puts an FCC
    # block at density 0.85 in the (more dilute) box, straddling a corner, so its
    # particles have more partners than the box's mean density predicts
    layout: str = "fcc"
    # filled in by the server
    admitted: float = math.nan
    finished: float = math.nan
    remaining: int = 0
    sid: int = -1
    active: bool = True
    result: dict = field(default_factory=dict)

    @property
    def box(self) -> float:
        return (self.n / self.rho) ** (1.0 / 3.0)


DROPLET_DENSITY = 0.85


def initial_state(r: Request):
    import lj_inputs as li
    if r.layout == "droplet":
        side = (r.n / DROPLET_DENSITY) ** (1.0 / 3.0)
        x = np.mod(li.fcc_positions(r.n, side) + (r.box - 0.5 * side), r.box)
    elif r.layout == "fcc":
        x = li.fcc_positions(r.n, r.box)
    else:
        raise ValueError(f"unknown layout {r.layout!r}")
    v = li.maxwell_boltzmann(r.n, r.temperature, r.seed)
    return x, v


class MDServer:
    """Admit, step and retire LJ runs in one arena. ``clock`` returns seconds."""

    def __init__(self, budget_bytes: int, precision: int = ljmd.MD_FP32_FORCE, chunk: int = 100,
                 max_systems: int = 4096, keep_state: bool = False, clock=time.perf_counter,
                 prepare_threads: int = 4, policy: str = "shared", active_particles: int = 2_500_000):
        """policy "shared": every admitted run advances in every chunk; "srpt": each
        chunk advances the runs with the least remaining work (particles x steps),
        smallest first, until `active_particles` are active (at least one run) and
        the others wait on the device. Pausing a run does not change its result."""
        if policy not in ("shared", "srpt"):
            raise ValueError("policy must be 'shared' or 'srpt'")
        self.policy = policy
        self.active_particles = int(active_particles)
        self.arena = arena_for_budget(budget_bytes, max_systems)
        # list words kept free at admission, so that admitted runs can grow their
        # lists (a denser region raises a run's partner count)
        self.list_reserve = self.arena["list_words"] // 20
        self.batch = ljmd.LJBatch(arena=self.arena, precision=precision)
        self.chunk = int(chunk)
        self.keep_state = keep_state
        self.clock = clock
        self.pending: collections.deque[Request] = collections.deque()
        self.running: dict[int, Request] = {}
        self.done: list[Request] = []
        self.particle_steps = 0
        self.gpu_busy = 0.0
        # initial states are generated on host threads as requests arrive, so that
        # admission only copies them to the device
        self.pool = cf.ThreadPoolExecutor(max_workers=prepare_threads)
        self.prepared: dict[int, cf.Future] = {}
        self.t0 = self.clock()  # times of requests are seconds since t0

    def close(self):
        self.pool.shutdown(wait=False, cancel_futures=True)
        self.batch.close()

    def fits_ever(self, r: Request) -> bool:
        f = ljmd.footprint(r.n, r.box, r.rc, r.skin)
        return (f["slots"] <= self.arena["slots"] and f["cells"] <= self.arena["cells"]
                and f["list_words"] <= self.arena["list_words"])

    def submit(self, r: Request):
        self.pending.append(r)
        self._prepare_ahead()

    def _prepare_ahead(self, depth: int = 32):
        """Start generating the states of the first `depth` pending requests."""
        for r in list(self.pending)[:depth]:
            if id(r) not in self.prepared:
                self.prepared[id(r)] = self.pool.submit(initial_state, r)

    def admit(self, now: float, backfill: int = 64):
        """FIFO admission; up to `backfill` later requests may pass a head that does
        not fit yet (smaller runs use the space it cannot)."""
        skipped = 0
        free_list = self.batch.usage()["list_words_free"]
        for r in list(self.pending):
            need = ljmd.footprint(r.n, r.box, r.rc, r.skin)["list_words"]
            sid = None
            if free_list - need >= self.list_reserve or not self.running:
                sid = self.batch.try_add(r.n, r.box, r.rc, r.skin)
            if sid is None:
                skipped += 1
                if skipped > backfill:
                    break
                continue
            free_list -= need
            fut = self.prepared.pop(id(r), None)
            x, v = fut.result() if fut is not None else initial_state(r)
            self.batch.set_state(sid, x, v)
            r.sid = sid
            r.admitted = now
            r.remaining = r.steps
            r.active = True
            self.running[sid] = r
            self.pending.remove(r)
        self._prepare_ahead()

    def _select_active(self) -> list[int]:
        """The runs to advance in this chunk (and set the others inactive)."""
        if self.policy == "shared":
            return list(self.running)
        order = sorted(self.running, key=lambda sid: (self.running[sid].n * self.running[sid].remaining, sid))
        active, total = [], 0
        for sid in order:
            if active and total >= self.active_particles:
                break
            active.append(sid)
            total += self.running[sid].n
        chosen = set(active)
        for sid, r in self.running.items():
            on = sid in chosen
            if r.active != on:
                self.batch.set_active(sid, on)
                r.active = on
        return active

    def cancel(self, r: Request, now: float):
        """Withdraw a request: drop it from the queue, or free its arena space if it
        is running (the other runs are not affected)."""
        if r in self.pending:
            self.pending.remove(r)
            fut = self.prepared.pop(id(r), None)
            if fut is not None:
                fut.cancel()
        elif r.sid in self.running and self.running[r.sid] is r:
            self.running.pop(r.sid)
            self.batch.remove(r.sid)
        else:
            return
        r.result = dict(cancelled=True)
        r.finished = now
        self.done.append(r)

    def _cancel_due(self, now: float):
        for r in [q for q in list(self.pending) + list(self.running.values())
                  if not math.isnan(q.cancel_after) and q.arrival + q.cancel_after <= now]:
            self.cancel(r, now)

    def step_chunk(self) -> int:
        if not self.running:
            return 0
        active = self._select_active()
        k = min(self.chunk, min(self.running[sid].remaining for sid in active))
        dts = {sid: r.dt for sid, r in self.running.items()}
        t = self.clock()
        self.batch.step(k, dts)
        self.gpu_busy += self.clock() - t
        finished = []
        for sid in active:
            r = self.running[sid]
            r.remaining -= k
            self.particle_steps += r.n * k
            if r.remaining == 0:
                finished.append(sid)
        if finished:
            obs = self.batch.observables(select=finished)
            now = self.clock() - self.t0
            for sid in finished:
                r = self.running.pop(sid)
                o = obs[sid]
                r.result = dict(pe=o[0], virial=o[1], ke=o[2], temperature=o[3], pressure=o[4],
                                rebuilds=self.batch.stats(sid)["rebuilds"])
                if self.keep_state:
                    r.result["x"], r.result["v"] = self.batch.get_state(sid)
                r.finished = now
                self.batch.remove(sid)
                self.done.append(r)
        return k

    def run(self, requests: list[Request], drain_limit: float | None = None) -> dict:
        """Replay requests at their arrival times (seconds from the start) in real
        time; stop when all are done or drain_limit seconds after the last arrival."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        self.t0 = t0 = self.clock()
        i = 0
        last_arrival = reqs[-1].arrival if reqs else 0.0
        while i < len(reqs) or self.pending or self.running:
            now = self.clock() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                r = reqs[i]
                i += 1
                if not self.fits_ever(r):
                    r.result = dict(rejected="larger than the whole arena")
                    r.finished = now
                    self.done.append(r)
                    continue
                self.submit(r)
            self._cancel_due(now)
            if self.pending:
                self.admit(now)
            if self.running:
                self.step_chunk()
            elif i < len(reqs):
                time.sleep(max(0.0, min(0.05, reqs[i].arrival - (self.clock() - t0))))
            if drain_limit is not None and now > last_arrival + drain_limit:
                break
        wall = self.clock() - t0
        return self.summary(reqs, wall)

    def summary(self, reqs: list[Request], wall: float) -> dict:
        done = [r for r in self.done if "rejected" not in r.result and "cancelled" not in r.result]
        lat = np.array([r.finished - r.arrival for r in done])
        wait = np.array([r.admitted - r.arrival for r in done])

        def pct(a, q):  # NaN when no request completed
            return float(np.percentile(a, q)) if a.size else math.nan

        done_ids = {id(r) for r in self.done}
        left = [r for r in reqs if id(r) not in done_ids]
        left_work = sum(r.n * (r.remaining if r.sid >= 0 and not math.isnan(r.admitted) else r.steps)
                        for r in left)
        rate = self.particle_steps / wall if wall > 0 else math.nan
        return dict(requests=len(reqs), completed=len(done),
                    rejected=sum(1 for r in self.done if "rejected" in r.result),
                    cancelled=sum(1 for r in self.done if "cancelled" in r.result),
                    unfinished=len(left), wall_s=wall,
                    p50_latency_s=pct(lat, 50),
                    p99_latency_s=pct(lat, 99),
                    p50_queue_s=pct(wait, 50),
                    p99_queue_s=pct(wait, 99),
                    particle_steps_per_s=rate,
                    gpu_busy_fraction=self.gpu_busy / wall if wall > 0 else math.nan,
                    remaining_particle_steps=int(left_work),
                    projected_drain_s=(left_work / rate) if rate and rate > 0 else math.nan)


def requests_from_workload(rate: float, duration: float, seed: int = 1005, **kw) -> list[Request]:
    import lj_inputs as li
    out = []
    for d in li.serve_requests(rate=rate, duration=duration, seed=seed, **kw):
        out.append(Request(id=d["id"], arrival=d["arrival"], n=d["n"], rho=d["rho"],
                           temperature=d["temperature"], steps=d["steps"], seed=d["seed"]))
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--duration", type=float, default=60.0)
    p.add_argument("--budget-gb", type=float, default=100.0)
    p.add_argument("--chunk", type=int, default=100)
    p.add_argument("--drain-limit", type=float, default=None)
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    a = p.parse_args(argv)
    from . import build
    build.build()
    reqs = requests_from_workload(a.rate, a.duration)
    srv = MDServer(int(a.budget_gb * 1e9), ljmd.MD_FP32_FORCE if a.precision == "fp32" else ljmd.MD_FP64,
                   chunk=a.chunk)
    try:
        s = srv.run(reqs, drain_limit=a.drain_limit)
    finally:
        srv.close()
    s.update(rate=a.rate, duration=a.duration, budget_gb=a.budget_gb, chunk=a.chunk)
    print(json.dumps(s))


if __name__ == "__main__":
    main()

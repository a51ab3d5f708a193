"""Seeded synthetic inputs for truncated-LJ molecular dynamics.

This module is shared by the CUDA path's tests and benchmarks and by the CPU
oracle's tests. It holds only input generation (lattice sites, random
displacements, random velocities, workload tables) and none of the method's
arithmetic: no potential, no force, no pair search, no integrator.

Random numbers come from numpy's PCG64 bit generator (O'Neill 2014,
"PCG: A Family of Simple Fast Space-Efficient Statistically Good Algorithms
for Random Number Generation"), through ``numpy.random.Generator``.

Recipes (reduced LJ units, m = sigma = epsilon = k_B = 1):

* face-centred-cubic start (Sec. 3.2 of the paper uses an FCC initial
  condition): the smallest ``n`` with ``4 n^3 >= N``; sites are enumerated
  in (ix, iy, iz, basis) lexicographic order and the first ``N`` are kept;
  lattice constant ``L / n``.
* Maxwell-Boltzmann velocities at temperature ``T``: standard normals,
  mean subtracted per axis, then rescaled so that ``2 KE / (3 (N - 1)) = T``.
* the paper's own benchmark velocities (Sec. 3.2): every particle has speed
  ``|v| = 0.9`` in a uniformly random direction.
* liquid-like positions for force parity: FCC sites displaced uniformly in
  ``[-a, a]^3``; with ``a <= 0.1`` at the densities used here no pair comes
  closer than about 0.85 sigma, as in a dense LJ liquid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "box_length", "fcc_positions", "maxwell_boltzmann", "fixed_speed_velocities",
    "perturbed_fcc", "uniform_positions", "MDConfig", "config_small_fluid",
    "config_large_fluid", "config_cavitation", "batch_systems", "serve_requests",
    "system_seed",
]


def box_length(n: int, rho: float) -> float:
    """Side of the cubic box holding ``n`` particles at number density ``rho``."""
    return (n / rho) ** (1.0 / 3.0)


_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_positions(n: int, box: float) -> np.ndarray:
    """First ``n`` FCC sites of an ``m^3``-cell lattice filling ``[0, box)^3``.

    Returns an ``(n, 3)`` float64 array (C order)."""
    m = 1
    while 4 * m ** 3 < n:
        m += 1
    a = box / m
    idx = np.arange(m)
    ix, iy, iz = np.meshgrid(idx, idx, idx, indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3)
    return np.ascontiguousarray(sites[:n] * a)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def maxwell_boltzmann(n: int, temperature: float, seed: int) -> np.ndarray:
    """Velocities with zero net momentum and exactly the requested temperature,
    where temperature is ``2 KE / (3 (n - 1))`` and ``KE = sum |v|^2 / 2``."""
    v = _rng(seed).standard_normal((n, 3))
    v -= v.mean(axis=0)
    if n > 1 and temperature > 0:
        ke = 0.5 * float(np.sum(v * v))
        v *= math.sqrt(temperature * 3.0 * (n - 1) / (2.0 * ke))
    else:
        v[:] = 0.0
    return np.ascontiguousarray(v)


def fixed_speed_velocities(n: int, speed: float, seed: int) -> np.ndarray:
    """Every particle gets speed ``speed`` in a uniformly random direction."""
    g = _rng(seed).standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return np.ascontiguousarray(g * speed)


def perturbed_fcc(n: int, rho: float, amplitude: float, seed: int) -> tuple[np.ndarray, float]:
    """FCC sites at density ``rho`` displaced uniformly in ``[-amplitude, amplitude]^3``,
    folded back into ``[0, box)`` with ``numpy.mod``. Returns ``(x, box)``."""
    box = box_length(n, rho)
    x = fcc_positions(n, box)
    x = x + _rng(seed).uniform(-amplitude, amplitude, size=x.shape)
    x = np.mod(x, box)
    x[x >= box] = 0.0
    return np.ascontiguousarray(x), box


def uniform_positions(n: int, box: float, seed: int) -> np.ndarray:
    """Independent uniform positions in ``[0, box)^3`` (overlaps allowed)."""
    return np.ascontiguousarray(_rng(seed).uniform(0.0, box, size=(n, 3)))


def system_seed(config_seed: int, index: int) -> int:
    """Per-system seed for multi-system workloads: splitmix64 finaliser of
    ``config_seed * 2^32 + index`` (Steele, Lea, Flood 2014, "Fast splittable
    pseudorandom number generators")."""
    z = (config_seed * (1 << 32) + index + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return int(z ^ (z >> 31))


@dataclass
class MDConfig:
    """One LJ system: box, cutoff, skin, time step and its initial state."""
    name: str
    n: int
    box: float
    rc: float
    skin: float
    dt: float
    steps: int
    x: np.ndarray = field(repr=False)
    v: np.ndarray = field(repr=False)
    rho: float = 0.0
    temperature: float = 0.0
    extra: dict = field(default_factory=dict)


def _fluid(name: str, cells: int, rho: float, temperature: float, rc: float, skin: float,
           dt: float, steps: int, seed: int) -> MDConfig:
    n = 4 * cells ** 3
    box = box_length(n, rho)
    x = fcc_positions(n, box)
    v = maxwell_boltzmann(n, temperature, seed)
    return MDConfig(name, n, box, rc, skin, dt, steps, x, v, rho, temperature)


def config_small_fluid() -> MDConfig:
    """N = 4000 (FCC 10^3 x 4), rho = 0.8442, T = 0.722, rc = 2.5, skin 0.3,
    dt = 0.005, 200 steps; seed 1001."""
    return _fluid("lj-fcc-4000-rho0.8442", 10, 0.8442, 0.722, 2.5, 0.3, 0.005, 200, 1001)


def config_large_fluid() -> MDConfig:
    """N = 2,048,000 (FCC 80^3 x 4), rho = 0.8442, T = 0.722, rc = 2.5, skin 0.3,
    dt = 0.005, 1000 steps; seed 1002."""
    return _fluid("lj-fcc-2048000-rho0.8442", 80, 0.8442, 0.722, 2.5, 0.3, 0.005, 1000, 1002)


def config_cavitation(cells: int = 160) -> MDConfig:
    """Cavitation-shaped start: N = 4 cells^3 (16,384,000 at 160 cells) at
    rho = 0.70, T = 0.90, rc = 3.0, skin 0.3, dt = 0.005, 20,000 NVE steps;
    seed 1003. The equilibration and the uniform expansion by 1.05 per axis are
    applied by the caller (they are part of the run protocol, not the input)."""
    cfg = _fluid(f"lj-cavitation-{4 * cells ** 3}-rho0.70", cells, 0.70, 0.90, 3.0, 0.3, 0.005,
                 20000, 1003)
    cfg.extra.update(expansion=1.05, equilibration_steps=2000, rescale_every=10)
    return cfg


def batch_systems(count: int = 256, seed: int = 1004, n_min: int = 500, n_max: int = 32000,
                  rho_range=(0.60, 0.85), t_range=(0.7, 1.2)) -> list[MDConfig]:
    """Independent replica systems: N log-uniform in [n_min, n_max], rho and T
    uniform in the given ranges, rc = 2.5, skin 0.3, dt = 0.005, 2000 steps.
    Positions are the first N FCC sites of the smallest lattice holding them."""
    out = []
    g = _rng(seed)
    ns = np.exp(g.uniform(math.log(n_min), math.log(n_max), size=count)).astype(np.int64)
    rhos = g.uniform(*rho_range, size=count)
    ts = g.uniform(*t_range, size=count)
    for k in range(count):
        n = int(ns[k])
        box = box_length(n, float(rhos[k]))
        x = fcc_positions(n, box)
        v = maxwell_boltzmann(n, float(ts[k]), system_seed(seed, k))
        out.append(MDConfig(f"replica-{k}", n, box, 2.5, 0.3, 0.005, 2000, x, v,
                            float(rhos[k]), float(ts[k])))
    return out


def serve_requests(rate: float = 200.0, duration: float = 60.0, seed: int = 1005,
                   n_range=(1_000, 1_000_000), rho_range=(0.6, 0.85), t_range=(0.722, 1.2),
                   steps_range=(1_000, 10_000)) -> list[dict]:
    """Poisson arrivals: list of request dicts with arrival time, N, rho, T and
    step count (states are generated on admission with ``system_seed``)."""
    g = _rng(seed)
    reqs = []
    t = 0.0
    k = 0
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        reqs.append(dict(id=k, arrival=t, n=n, rho=float(g.uniform(*rho_range)),
                         temperature=float(g.uniform(*t_range)),
                         steps=int(g.integers(steps_range[0], steps_range[1] + 1)),
                         seed=system_seed(seed, k)))
        k += 1
    return reqs

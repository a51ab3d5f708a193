"""Plain FP64 CPU oracle for truncated-LJ molecular dynamics (ctypes wrapper).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only the test suite, the
package's smoke check and the benchmark's CPU-baseline leg use it. It shares
no code with the CUDA path and never imports it.

Every function follows the paper (Watanabe, Suzuki, Ito, arXiv:1210.3450):
Eq. 1 for the truncated potential, Sec. 2.1 for the cell search and the
bookkeeping list, Algorithm 1 (Sec. 3.3) for the full-list force factor, and
the second-order symplectic (velocity Verlet) update of Sec. 3.2 / 4.1.
The arithmetic lives in ``ljmd_oracle.c``; this module only marshals arrays.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build as _build

_lib = None

_D = C.c_double
_I64 = C.c_int64
_PD = C.POINTER(C.c_double)
_PI64 = C.POINTER(C.c_int64)
_PI32 = C.POINTER(C.c_int32)


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(_build())
        sig = {
            "orc_lj_coeffs": (None, [_D, _PD, _PD]),
            "orc_pair_energy": (_D, [_D, _D, _D, _D]),
            "orc_pair_force_factor": (_D, [_D, _D, _D]),
            "orc_pair_virial": (_D, [_D, _D, _D]),
            "orc_wrap": (None, [_I64, _D, _PD]),
            "orc_cells_per_axis": (C.c_int, [_D, _D]),
            "orc_cell_index": (None, [_I64, _D, C.c_int, _PD, _PI32]),
            "orc_build_list": (_I64, [_I64, _D, _D, _PD, _PI64, _PI32, _I64]),
            "orc_build_list_brute": (_I64, [_I64, _D, _D, _PD, _PI64, _PI32, _I64]),
            "orc_forces_list": (None, [_I64, _D, _D, _D, _PD, _PI64, _PI32, _PD]),
            "orc_force_on": (None, [_I64, _D, _D, _D, _PD, _I64, _PD]),
            "orc_forces_brute": (None, [_I64, _D, _D, _D, _PD, _PD]),
            "orc_observables_list": (None, [_I64, _D, _D, _D, _D, _PD, _PD, _PI64, _PI32, _PD]),
            "orc_forces_half": (None, [_I64, _D, _D, _D, _PD, _PI64, _PI32, _PD]),
            "orc_run": (C.c_int, [_I64, _D, _D, _D, _PD, _PD, _I64, _D, _PI64, _PD, _I64]),
            "orc_run_mode": (C.c_int, [_I64, _D, _D, _D, _PD, _PD, _I64, _D, _PI64, _PD, _I64,
                                       C.c_int, C.c_int]),
            "orc_run_rule": (C.c_int, [_I64, _D, _D, _D, _PD, _PD, _I64, _D, _PI64, _PD, _I64,
                                       C.c_int, C.c_int, C.c_int]),
            "orc_pair_force_factor_rcp": (_D, [_D, _D, _D, C.c_int, C.c_int]),
            "orc_subcell_counts": (None, [_I64, _D, C.c_int, _PD, _PI32]),
            "orc_run_nvt": (C.c_int, [_I64, _D, _D, _D, _PD, _PD, _I64, _D, _D, _D, _PD, _PI64, _PD, _I64]),
            "orc_clusters": (_I64, [C.c_int, C.POINTER(C.c_uint8), _PI32]),
            "orc_forces_list_rcp": (None, [_I64, _D, _D, _D, _PD, _PI64, _PI32, C.c_int, C.c_int, _PD]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _pd(a):
    return a.ctypes.data_as(_PD)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def lj_coeffs(rc: float) -> tuple[float, float]:
    """(c2, c0) of Eq. 1 from V(rc) = V'(rc) = 0."""
    c2, c0 = _D(), _D()
    _load().orc_lj_coeffs(rc, C.byref(c2), C.byref(c0))
    return c2.value, c0.value


def pair_energy(r2: float, rc: float, c2: float, c0: float) -> float:
    return _load().orc_pair_energy(r2, rc * rc, c2, c0)


def pair_force_factor(r2: float, rc: float, c2: float) -> float:
    return _load().orc_pair_force_factor(r2, rc * rc, c2)


def pair_virial(r2: float, rc: float, c2: float) -> float:
    return _load().orc_pair_virial(r2, rc * rc, c2)


def wrap(x, box: float) -> np.ndarray:
    x = _f64(x, (-1, 3)).copy()
    _load().orc_wrap(x.shape[0], box, _pd(x))
    return x


def cells_per_axis(box: float, rl: float) -> int:
    return _load().orc_cells_per_axis(box, rl)


def cell_index(x, box: float, rl: float) -> np.ndarray:
    """Linear cell index cx + nc (cy + nc cz) of each particle (positions in [0, L))."""
    x = _f64(x, (-1, 3))
    nc = cells_per_axis(box, rl)
    out = np.empty(x.shape[0], dtype=np.int32)
    _load().orc_cell_index(x.shape[0], box, nc, _pd(x), out.ctypes.data_as(_PI32))
    return out


def build_list(x, box: float, rl: float, brute: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Full list {j != i : min-image r^2 < rl^2}: (start[n+1] int64, partners int32),
    partners of each i ascending."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    start = np.empty(n + 1, dtype=np.int64)
    cap = max(64, n * 96)
    fn = _load().orc_build_list_brute if brute else _load().orc_build_list
    while True:
        partners = np.empty(cap, dtype=np.int32)
        got = fn(n, box, rl, _pd(x), start.ctypes.data_as(_PI64), partners.ctypes.data_as(_PI32), cap)
        if got >= 0:
            return start, partners[:got].copy()
        cap = -got


def forces_list(x, box: float, rc: float, c2: float, start, partners) -> np.ndarray:
    x = _f64(x, (-1, 3))
    f = np.empty_like(x)
    start = np.ascontiguousarray(start, dtype=np.int64)
    partners = np.ascontiguousarray(partners, dtype=np.int32)
    _load().orc_forces_list(x.shape[0], box, rc, c2, _pd(x), start.ctypes.data_as(_PI64),
                            partners.ctypes.data_as(_PI32), _pd(f))
    return f


def forces_half(x, box: float, rc: float, skin: float = 0.3) -> np.ndarray:
    """Forces with Newton's third law: each pair i < j of the list once, +g r on i
    and -g r on j."""
    x = _f64(x, (-1, 3))
    start, partners = build_list(x, box, rc + skin)
    c2, _ = lj_coeffs(rc)
    f = np.empty_like(x)
    _load().orc_forces_half(x.shape[0], box, rc, c2, _pd(x), np.ascontiguousarray(start).ctypes.data_as(_PI64),
                            np.ascontiguousarray(partners, dtype=np.int32).ctypes.data_as(_PI32), _pd(f))
    return f


def pair_force_factor_rcp(r2: float, rc: float, c2: float, bits: int, corr: bool) -> float:
    """Force factor with r^-8, r^-14 from an approximate reciprocal of r^2 (Sec. 3.3,
    Eqs. 2-7): `bits` mantissa bits kept (8: relative error < 1/256), corrected or not."""
    return _load().orc_pair_force_factor_rcp(r2, rc * rc, c2, int(bits), 1 if corr else 0)


def forces_rcp(x, box: float, rc: float, bits: int, corr: bool, skin: float = 0.3) -> np.ndarray:
    c2 = lj_coeffs(rc)[0]
    x = _f64(x, (-1, 3))
    start, partners = build_list(x, box, rc + skin)
    f = np.empty_like(x)
    _load().orc_forces_list_rcp(x.shape[0], box, rc, c2, _pd(x), start.ctypes.data_as(_PI64),
                                partners.ctypes.data_as(_PI32), int(bits), 1 if corr else 0, _pd(f))
    return f


def forces(x, box: float, rc: float, skin: float = 0.3, c2: float | None = None) -> np.ndarray:
    """Forces through the cell-built list (list radius rc + skin)."""
    if c2 is None:
        c2 = lj_coeffs(rc)[0]
    start, partners = build_list(x, box, rc + skin)
    return forces_list(x, box, rc, c2, start, partners)


def forces_brute(x, box: float, rc: float, c2: float | None = None) -> np.ndarray:
    if c2 is None:
        c2 = lj_coeffs(rc)[0]
    x = _f64(x, (-1, 3))
    f = np.empty_like(x)
    _load().orc_forces_brute(x.shape[0], box, rc, c2, _pd(x), _pd(f))
    return f


def force_on(x, box: float, rc: float, i: int, c2: float | None = None) -> np.ndarray:
    """Force on one particle by direct summation over all others."""
    if c2 is None:
        c2 = lj_coeffs(rc)[0]
    x = _f64(x, (-1, 3))
    out = np.empty(3)
    _load().orc_force_on(x.shape[0], box, rc, c2, _pd(x), int(i), _pd(out))
    return out


def observables(x, v, box: float, rc: float, skin: float = 0.3, c2=None, c0=None) -> dict:
    """PE, virial W, KE, T = 2KE/(3(N-1)), P = (2KE + W)/(3V)."""
    if c2 is None or c0 is None:
        c2, c0 = lj_coeffs(rc)
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    start, partners = build_list(x, box, rc + skin)
    out = np.empty(5)
    _load().orc_observables_list(x.shape[0], box, rc, c2, c0, _pd(x), _pd(v),
                                 start.ctypes.data_as(_PI64), partners.ctypes.data_as(_PI32),
                                 _pd(out))
    return dict(pe=out[0], virial=out[1], ke=out[2], temperature=out[3], pressure=out[4])


def run(x, v, box: float, rc: float, skin: float, nsteps: int, dt: float,
        trace_every: int = 0, rcp_bits: int = -1, rcp_corr: bool = False, rule: int = 0) -> dict:
    """Velocity-Verlet run; returns dict(x, v, rebuilds, trace). With rcp_bits >= 0 the
    forces use the approximate-reciprocal factor of Sec. 3.3; rule 1 checks the list
    with the velocity bound (DUTC) instead of the displacements."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    rebuilds = _I64(0)
    trace = None
    tp = None
    if trace_every > 0:
        trace = np.empty(1 + nsteps // trace_every)
        tp = _pd(trace)
    rc_ = _load().orc_run_rule(x.shape[0], box, rc, skin, _pd(x), _pd(v), nsteps, dt,
                               C.byref(rebuilds), tp, trace_every, int(rcp_bits), 1 if rcp_corr else 0,
                               int(rule))
    if rc_ != 0:
        raise MemoryError("oracle run failed to allocate")
    return dict(x=x, v=v, rebuilds=rebuilds.value, trace=trace)


def subcell_counts(x, box: float, side: float = 3.0) -> tuple[np.ndarray, int]:
    """Particles per subcell (Sec. 4.2), ns = floor(L / side) subcells per axis."""
    x = _f64(x, (-1, 3))
    ns = max(1, int(np.floor(box / side)))
    counts = np.empty(ns ** 3, dtype=np.int32)
    _load().orc_subcell_counts(x.shape[0], box, ns, _pd(x), counts.ctypes.data_as(_PI32))
    return counts, ns


def clusters(gas, ns: int) -> tuple[int, np.ndarray]:
    """Face-connected clusters of gas subcells on the periodic ns^3 lattice:
    (number of clusters, label per subcell = smallest index of its cluster or -1)."""
    g = np.ascontiguousarray(np.asarray(gas, dtype=np.uint8).reshape(-1))
    label = np.empty(ns ** 3, dtype=np.int32)
    k = _load().orc_clusters(ns, g.ctypes.data_as(C.POINTER(C.c_uint8)), label.ctypes.data_as(_PI32))
    return int(k), label


def bubbles(x, box: float, side: float = 3.0, gas_density: float = 0.2) -> dict:
    """Bubble identification of Sec. 4.2: subcell counts, gas where the density is
    below gas_density, clusters by site percolation; sizes in subcells, descending."""
    counts, ns = subcell_counts(x, box, side)
    vol = (box / ns) ** 3
    gas = counts.astype(np.float64) < gas_density * vol
    k, label = clusters(gas, ns)
    sizes = np.bincount(label[label >= 0]) if k else np.zeros(0, dtype=np.int64)
    sizes = np.sort(sizes[sizes > 0])[::-1]
    return dict(ns=ns, counts=counts, gas=gas, n_bubbles=k, sizes=sizes, label=label)


def run_nvt(x, v, box: float, rc: float, skin: float, nsteps: int, dt: float, temperature: float,
            q: float, zeta: float = 0.0, eta: float = 0.0, trace_every: int = 0) -> dict:
    """Nose-Hoover NVT run (Sec. 4.1 thermostat; reversible splitting: thermostat half
    step, velocity-Verlet step, thermostat half step). Returns dict(x, v, zeta, eta,
    trace) where trace is KE + PE + Q zeta^2/2 + g T eta (the conserved quantity)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    ze = np.array([zeta, eta], dtype=np.float64)
    rebuilds = _I64(0)
    trace = None
    tp = None
    if trace_every > 0:
        trace = np.empty(1 + nsteps // trace_every)
        tp = _pd(trace)
    r = _load().orc_run_nvt(x.shape[0], box, rc, skin, _pd(x), _pd(v), nsteps, dt, temperature, q,
                            _pd(ze), C.byref(rebuilds), tp, trace_every)
    if r != 0:
        raise MemoryError("oracle run failed")
    return dict(x=x, v=v, zeta=float(ze[0]), eta=float(ze[1]), trace=trace, rebuilds=rebuilds.value)

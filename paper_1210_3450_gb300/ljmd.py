"""Python binding of the C ABI in ``include/ljmd.h`` (ctypes; argument
marshalling only). Every computation runs in the CUDA library
``_build/libljmd.so``; there is no CPU fallback: loading fails loudly if the
library is missing or cannot be loaded.

Host-array calls take numpy arrays of shape (N, 3), float64. The ``*_dev``
calls take CUDA torch tensors (float64, contiguous) and an optional
``torch.cuda.Stream``; torch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

MD_OK = 0
MD_ERR_ARG = -1
MD_ERR_OOM = -2
MD_ERR_LIST_OVERFLOW = -3
MD_ERR_NONFINITE = -4
MD_ERR_TIMEOUT = -5
MD_ERR_CUDA = -6
MD_ERR_STATE = -7
MD_ERR_CHECK = -8
MD_FP64 = 0
MD_FP32_FORCE = 1
MD_FP64_RCP8 = 2
MD_FP64_RCP8_CORR = 3
MD_FP64_RCP23 = 4
MD_FP64_RCP23_CORR = 5
MD_MAX_N = (1 << 26) - 1
MD_RULE_DISPLACEMENT = 0
MD_RULE_DUTC = 1
MD_LIST_FULL = 0
MD_LIST_HALF = 1
MD_TUNE_STEP_BLOCK = 0
MD_TUNE_STEP_GROUPS = 1
MD_TUNE_LIST_BLOCK = 2
MD_TUNE_LIST_VARIANT = 3
MD_TUNE_STEP_HINT = 4
MD_TUNE_GRAPH = 5
MD_TUNE_FP64_QUEUE = 6
TUNING_KEYS = {"step_block": MD_TUNE_STEP_BLOCK, "step_groups": MD_TUNE_STEP_GROUPS,
               "list_block": MD_TUNE_LIST_BLOCK, "list_variant": MD_TUNE_LIST_VARIANT,
               "step_hint": MD_TUNE_STEP_HINT, "graph": MD_TUNE_GRAPH, "fp64_queue": MD_TUNE_FP64_QUEUE}

_ERRNAMES = {v: k for k, v in dict(MD_ERR_ARG=-1, MD_ERR_OOM=-2, MD_ERR_LIST_OVERFLOW=-3,
                                   MD_ERR_NONFINITE=-4, MD_ERR_TIMEOUT=-5, MD_ERR_CUDA=-6,
                                   MD_ERR_STATE=-7, MD_ERR_CHECK=-8).items()}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libljmd.so")
# the same library with device bounds checks (a test and debugging tool)
CHECKED_LIB_PATH = os.path.join(_HERE, "_build", "checked", "libljmd.so")

_lib = None
_P = C.c_void_p
_PD = C.POINTER(C.c_double)
_PI64 = C.POINTER(C.c_int64)
_PI32 = C.POINTER(C.c_int32)

# name -> (restype, argtypes); mirrors include/ljmd.h
SIGNATURES = {
    "md_create": (C.c_int, [C.c_double, C.c_int64, C.c_double, C.c_double, C.POINTER(_P)]),
    "md_set_precision": (C.c_int, [_P, C.c_int]),
    "md_set_validity_rule": (C.c_int, [_P, C.c_int]),
    "md_get_checkpoint": (C.c_int, [_P, _PD, _PD, _PD, C.POINTER(C.c_double)]),
    "md_set_checkpoint": (C.c_int, [_P, _PD, _PD, _PD, C.c_double]),
    "md_set_pair_list": (C.c_int, [_P, C.c_int]),
    "md_set_state": (C.c_int, [_P, _PD, _PD]),
    "md_set_state_dev": (C.c_int, [_P, _P, _P, _P]),
    "md_get_state": (C.c_int, [_P, _PD, _PD]),
    "md_get_state_dev": (C.c_int, [_P, _P, _P, _P]),
    "md_step": (C.c_int, [_P, C.c_int64, C.c_double]),
    "md_step_async": (C.c_int, [_P, C.c_int64, C.c_double, _P]),
    "md_forces": (C.c_int, [_P, _PD]),
    "md_step_nvt": (C.c_int, [_P, C.c_int64, C.c_double, C.c_double, C.c_double, _PD, _PD]),
    "md_batch_step_nvt": (C.c_int, [_P, C.c_int64, _PD, _PD, _PD, _PD, _PD]),
    "md_forces_dev": (C.c_int, [_P, _P, _P]),
    "md_observables": (C.c_int, [_P, _PD, _PD, _PD, _PD, _PD]),
    "md_stats": (C.c_int, [_P, _PI64, _PI64]),
    "md_kinetic_energy": (C.c_int, [_P, _PD]),
    "md_scale_velocities": (C.c_int, [_P, C.c_double]),
    "md_batch_kinetic_energy": (C.c_int, [_P, _PD]),
    "md_batch_scale_velocities": (C.c_int, [_P, _PD]),
    "md_build_list": (C.c_int, [_P]),
    "md_get_cells": (C.c_int, [_P, _PI32, _PI32]),
    "md_list_size": (C.c_int, [_P, _PI64]),
    "md_batch_get_checkpoint": (C.c_int, [_P, C.c_int, _PD, _PD, _PD, _PD]),
    "md_batch_set_checkpoint": (C.c_int, [_P, C.c_int, _PD, _PD, _PD, C.c_double]),
    "md_debug_set_list_word": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_uint32]),
    "md_get_list": (C.c_int, [_P, _PI64, _PI32]),
    "md_pair_stats": (C.c_int, [_P, _PI64, _PI64]),
    "md_bubbles": (C.c_int, [_P, C.c_double, C.c_double, _PI32, C.POINTER(C.c_uint8), _PI64, _PI64, C.c_int64]),
    "md_set_timing": (C.c_int, [_P, C.c_int]),
    "md_get_timing": (C.c_int, [_P, _PD]),
    "md_forces_noalloc": (C.c_int, [_P, C.c_int64, C.c_double, C.c_double, _P, _P]),
    "md_probe_fma_rate": (C.c_int, [C.c_int, C.c_int64, _PD]),
    "md_set_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "md_get_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "md_batch_set_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "md_batch_get_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "md_destroy": (None, [_P]),
    "md_batch_create": (C.c_int, [C.c_int, _P, C.c_int, C.POINTER(_P)]),
    "md_batch_create_arena": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, C.POINTER(_P)]),
    "md_batch_footprint": (C.c_int, [_P, _PI64, _PI64, _PI64]),
    "md_batch_add": (C.c_int, [_P, _P, C.POINTER(C.c_int)]),
    "md_batch_remove": (C.c_int, [_P, C.c_int]),
    "md_batch_usage": (C.c_int, [_P, _PI64]),
    "md_batch_set_active": (C.c_int, [_P, C.c_int, C.c_int]),
    "md_batch_set_precision": (C.c_int, [_P, C.c_int]),
    "md_batch_set_validity_rule": (C.c_int, [_P, C.c_int]),
    "md_batch_set_pair_list": (C.c_int, [_P, C.c_int]),
    "md_batch_set_state": (C.c_int, [_P, C.c_int, _PD, _PD]),
    "md_batch_set_state_dev": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "md_batch_get_state": (C.c_int, [_P, C.c_int, _PD, _PD]),
    "md_batch_get_state_dev": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "md_batch_step": (C.c_int, [_P, C.c_int64, _PD]),
    "md_batch_step_async": (C.c_int, [_P, C.c_int64, _PD, _P]),
    "md_batch_forces": (C.c_int, [_P, C.c_int, _PD]),
    "md_batch_observables": (C.c_int, [_P, _PD]),
    "md_batch_observables_select": (C.c_int, [_P, _PI32, _PD]),
    "md_batch_stats": (C.c_int, [_P, C.c_int, _PI64, _PI64]),
    "md_batch_set_timing": (C.c_int, [_P, C.c_int]),
    "md_batch_get_timing": (C.c_int, [_P, _PD]),
    "md_batch_destroy": (None, [_P]),
    "md_last_error": (C.c_char_p, []),
    "md_version": (C.c_char_p, []),
}


class MDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def load_library(path: str | None = None):
    """Load (once) the CUDA library; raises if it is not built or not loadable."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libljmd is not built ({path} missing); run paper_1210_3450_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int):
    if code != MD_OK:
        raise MDError(code, _lib.md_last_error().decode())


def _host3(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)
    if a.shape[0] != n:
        raise ValueError(f"expected {n} rows, got {a.shape[0]}")
    return a


def _out3(out, n: int):
    """Caller-provided (x, v) output arrays (C-contiguous float64, n x 3), or new ones."""
    if out is None:
        return np.empty((n, 3)), np.empty((n, 3))
    x, v = out
    for a in (x, v):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.shape == (n, 3)):
            raise ValueError(f"output arrays must be C-contiguous float64 of shape ({n}, 3)")
    return x, v


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def _dev_ptr(t, n: int) -> int:
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64" and t.numel() == 3 * n):
        raise ValueError("expected a contiguous CUDA float64 tensor with N*3 elements")
    return int(t.data_ptr())


class LJSystem:
    """One periodic truncated-LJ system on the current CUDA device (md_create)."""

    def __init__(self, box: float, n: int, rc: float, skin: float, precision: int = MD_FP64):
        lib = load_library()
        h = _P()
        _check(lib.md_create(float(box), int(n), float(rc), float(skin), C.byref(h)))
        self._h = h
        self.n = int(n)
        self.box = float(box)
        self.rc = float(rc)
        self.skin = float(skin)
        if precision != MD_FP64:
            self.set_precision(precision)

    # lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # C ABI calls
    def set_precision(self, mode: int):
        _check(_lib.md_set_precision(self._h, int(mode)))

    def set_validity_rule(self, rule: int):
        _check(_lib.md_set_validity_rule(self._h, int(rule)))

    def set_pair_list(self, kind: int):
        _check(_lib.md_set_pair_list(self._h, int(kind)))

    def checkpoint(self) -> dict:
        """Exact checkpoint: positions as held (not wrapped), velocities, positions at
        the last list build, velocity-bound margin."""
        x = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        xb = np.empty((self.n, 3))
        m = C.c_double()
        _check(_lib.md_get_checkpoint(self._h, _pd(x), _pd(v), _pd(xb), C.byref(m)))
        return dict(x=x, v=v, x_build=xb, margin=m.value)

    def restore(self, ck: dict):
        """Restore a checkpoint taken from a system with the same sizes and settings."""
        x = _host3(ck["x"], self.n)
        v = _host3(ck["v"], self.n)
        xb = _host3(ck["x_build"], self.n)
        _check(_lib.md_set_checkpoint(self._h, _pd(x), _pd(v), _pd(xb), float(ck["margin"])))

    def set_state(self, x, v):
        x = _host3(x, self.n)
        v = _host3(v, self.n)
        _check(_lib.md_set_state(self._h, _pd(x), _pd(v)))

    def set_state_dev(self, x, v, stream=None):
        _check(_lib.md_set_state_dev(self._h, _dev_ptr(x, self.n), _dev_ptr(v, self.n), _stream_ptr(stream)))

    def get_state(self, out=None):
        """Positions (wrapped into [0, L)) and velocities in caller order; `out`
        may give the (x, v) arrays to fill, e.g. views of pinned host memory."""
        x, v = _out3(out, self.n)
        _check(_lib.md_get_state(self._h, _pd(x), _pd(v)))
        return x, v

    def get_state_dev(self, x=None, v=None, stream=None):
        _check(_lib.md_get_state_dev(self._h, _dev_ptr(x, self.n) if x is not None else None,
                                     _dev_ptr(v, self.n) if v is not None else None,
                                     _stream_ptr(stream)))

    def step(self, nsteps: int, dt: float):
        _check(_lib.md_step(self._h, int(nsteps), float(dt)))

    def step_async(self, nsteps: int, dt: float, stream=None):
        _check(_lib.md_step_async(self._h, int(nsteps), float(dt), _stream_ptr(stream)))

    def forces(self) -> np.ndarray:
        f = np.empty((self.n, 3))
        _check(_lib.md_forces(self._h, _pd(f)))
        return f

    def step_nvt(self, nsteps: int, dt: float, temperature: float, q: float, zeta: float = 0.0,
                 eta: float = 0.0) -> tuple[float, float]:
        """Nose-Hoover NVT steps (md_step_nvt); returns the updated (zeta, eta)."""
        z, e = C.c_double(zeta), C.c_double(eta)
        _check(_lib.md_step_nvt(self._h, int(nsteps), float(dt), float(temperature), float(q),
                                C.byref(z), C.byref(e)))
        return z.value, e.value

    def forces_dev(self, f, stream=None):
        _check(_lib.md_forces_dev(self._h, _dev_ptr(f, self.n), _stream_ptr(stream)))

    def observables(self) -> dict:
        vals = [C.c_double() for _ in range(5)]
        _check(_lib.md_observables(self._h, *[C.byref(v) for v in vals]))
        return dict(zip(["pe", "virial", "ke", "temperature", "pressure"], [v.value for v in vals]))

    def stats(self) -> dict:
        r, s = C.c_int64(), C.c_int64()
        _check(_lib.md_stats(self._h, C.byref(r), C.byref(s)))
        return dict(rebuilds=r.value, steps=s.value)

    def kinetic_energy(self) -> float:
        ke = C.c_double()
        _check(_lib.md_kinetic_energy(self._h, C.byref(ke)))
        return ke.value

    def scale_velocities(self, factor: float):
        _check(_lib.md_scale_velocities(self._h, float(factor)))

    def build_list(self):
        _check(_lib.md_build_list(self._h))

    def get_cells(self) -> tuple[np.ndarray, int]:
        cell = np.empty(self.n, dtype=np.int32)
        nc = C.c_int32()
        _check(_lib.md_get_cells(self._h, cell.ctypes.data_as(_PI32), C.byref(nc)))
        return cell, nc.value

    def debug_set_list_word(self, slot: int, entry: int, word: int):
        """Checked build only: overwrite one raw list word (a test of the device checks)."""
        _check(_lib.md_debug_set_list_word(self._h, int(slot), int(entry), int(word) & 0xFFFFFFFF))

    def list_size(self) -> int:
        t = C.c_int64()
        _check(_lib.md_list_size(self._h, C.byref(t)))
        return t.value

    def pair_stats(self) -> tuple[int, int]:
        """(listed pairs, listed pairs with r < rc at the current positions)."""
        a, b = C.c_int64(), C.c_int64()
        _check(_lib.md_pair_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_timing(self, on: bool = True):
        _check(_lib.md_set_timing(self._h, 1 if on else 0))

    def bubbles(self, side: float = 3.0, gas_density: float = 0.2) -> dict:
        """Bubble identification of Sec. 4.2 (md_bubbles): ns, uint8 subcell counts,
        number of bubbles and their sizes in subcells (descending)."""
        ns = max(1, int(np.floor(self.box / side)))
        counts = np.empty(ns ** 3, dtype=np.uint8)
        nb = C.c_int64()
        nsr = C.c_int32()
        cap = ns ** 3
        sizes = np.empty(cap, dtype=np.int64)
        _check(_lib.md_bubbles(self._h, float(side), float(gas_density), C.byref(nsr),
                               counts.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(nb),
                               sizes.ctypes.data_as(_PI64), cap))
        return dict(ns=nsr.value, counts=counts, n_bubbles=nb.value, sizes=sizes[:nb.value].copy())

    def set_tuning(self, **kw):
        for k, v in kw.items():
            _check(_lib.md_set_tuning(self._h, TUNING_KEYS[k], int(v)))

    def get_tuning(self) -> dict:
        out = {}
        for k, key in TUNING_KEYS.items():
            v = C.c_int()
            _check(_lib.md_get_tuning(self._h, key, C.byref(v)))
            out[k] = v.value
        return out

    def get_timing(self) -> dict:
        out = np.zeros(8)
        _check(_lib.md_get_timing(self._h, _pd(out)))
        return dict(step_ms=out[0], step_launches=int(out[1]), list_ms=out[2],
                    list_launches=int(out[3]), bin_ms=out[4], rebuilds=int(out[5]),
                    launches=int(out[6]))

    def get_list(self) -> tuple[np.ndarray, np.ndarray]:
        total = self.list_size()
        start = np.empty(self.n + 1, dtype=np.int64)
        partners = np.empty(max(total, 1), dtype=np.int32)
        _check(_lib.md_get_list(self._h, start.ctypes.data_as(_PI64), partners.ctypes.data_as(_PI32)))
        return start, partners[:total]


class SysDesc(C.Structure):
    """md_sys_desc: one system of a batch."""
    _fields_ = [("N", C.c_int64), ("box_L", C.c_double), ("rc", C.c_double), ("skin", C.c_double)]


def footprint(n: int, box: float, rc: float, skin: float) -> dict:
    """Arena space one system needs (md_batch_footprint)."""
    d = SysDesc(int(n), float(box), float(rc), float(skin))
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load_library().md_batch_footprint(C.byref(d), C.byref(a), C.byref(b), C.byref(c)))
    return dict(slots=a.value, cells=b.value, list_words=c.value)


class LJBatch:
    """Many independent LJ systems in one device arena (md_batch_*). Either a
    fixed set (``systems=[(n, box, rc, skin), ...]``, ids 0..k-1) or an empty
    arena with capacities (``arena=dict(slots=, cells=, list_words=, max_systems=)``)
    that systems are added to and removed from."""

    def __init__(self, systems=None, arena=None, precision: int = MD_FP64):
        lib = load_library()
        h = _P()
        if systems is not None:
            descs = (SysDesc * len(systems))(*[SysDesc(int(n), float(b), float(rc), float(sk))
                                               for (n, b, rc, sk) in systems])
            _check(lib.md_batch_create(len(systems), C.cast(descs, _P), int(precision), C.byref(h)))
            self.max_systems = len(systems)
            self._n = {k: int(systems[k][0]) for k in range(len(systems))}
        else:
            a = arena
            _check(lib.md_batch_create_arena(int(a["slots"]), int(a["cells"]), int(a["list_words"]),
                                             int(a["max_systems"]), int(precision), C.byref(h)))
            self.max_systems = int(a["max_systems"])
            self._n = {}
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.md_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, n: int, box: float, rc: float, skin: float) -> int:
        d = SysDesc(int(n), float(box), float(rc), float(skin))
        i = C.c_int()
        _check(_lib.md_batch_add(self._h, C.byref(d), C.byref(i)))
        self._n[i.value] = int(n)
        return i.value

    def try_add(self, n: int, box: float, rc: float, skin: float):
        """add(), or None when the arena has no room (MD_ERR_OOM)."""
        try:
            return self.add(n, box, rc, skin)
        except MDError as e:
            if e.code == MD_ERR_OOM:
                return None
            raise

    def remove(self, sid: int):
        _check(_lib.md_batch_remove(self._h, int(sid)))
        self._n.pop(sid, None)

    def usage(self) -> dict:
        o = np.zeros(8, dtype=np.int64)
        _check(_lib.md_batch_usage(self._h, o.ctypes.data_as(_PI64)))
        keys = ["slots", "slots_free", "cells", "cells_free", "list_words", "list_words_free",
                "systems", "systems_used"]
        return dict(zip(keys, [int(v) for v in o]))

    def set_active(self, sid: int, on: bool):
        _check(_lib.md_batch_set_active(self._h, int(sid), 1 if on else 0))

    def set_precision(self, mode: int):
        _check(_lib.md_batch_set_precision(self._h, int(mode)))

    def set_validity_rule(self, rule: int):
        _check(_lib.md_batch_set_validity_rule(self._h, int(rule)))

    def set_pair_list(self, kind: int):
        _check(_lib.md_batch_set_pair_list(self._h, int(kind)))

    def set_state(self, sid: int, x, v):
        n = self._n[sid]
        x = _host3(x, n)
        v = _host3(v, n)
        _check(_lib.md_batch_set_state(self._h, int(sid), _pd(x), _pd(v)))

    def set_state_dev(self, sid: int, x, v, stream=None):
        n = self._n[sid]
        _check(_lib.md_batch_set_state_dev(self._h, int(sid), _dev_ptr(x, n), _dev_ptr(v, n),
                                           _stream_ptr(stream)))

    def get_state(self, sid: int, out=None):
        x, v = _out3(out, self._n[sid])
        _check(_lib.md_batch_get_state(self._h, int(sid), _pd(x), _pd(v)))
        return x, v

    def checkpoint(self, sid: int) -> dict:
        """Exact checkpoint of system sid (see LJSystem.checkpoint)."""
        n = self._n[sid]
        x, v, xb = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
        m = C.c_double()
        _check(_lib.md_batch_get_checkpoint(self._h, int(sid), _pd(x), _pd(v), _pd(xb), C.byref(m)))
        return dict(x=x, v=v, x_build=xb, margin=m.value)

    def restore(self, sid: int, ck: dict):
        """Restore a checkpoint into system sid (same sizes and settings)."""
        n = self._n[sid]
        x, v, xb = _host3(ck["x"], n), _host3(ck["v"], n), _host3(ck["x_build"], n)
        _check(_lib.md_batch_set_checkpoint(self._h, int(sid), _pd(x), _pd(v), _pd(xb), float(ck["margin"])))

    def get_state_dev(self, sid: int, x=None, v=None, stream=None):
        """Positions and velocities of system sid into CUDA tensors (caller order)."""
        n = self._n[sid]
        _check(_lib.md_batch_get_state_dev(self._h, int(sid), _dev_ptr(x, n) if x is not None else None,
                                           _dev_ptr(v, n) if v is not None else None, _stream_ptr(stream)))

    def _dt(self, dt):
        arr = np.zeros(self.max_systems)
        if np.isscalar(dt):
            arr[:] = float(dt)
        elif isinstance(dt, dict):
            for k, val in dt.items():
                arr[k] = val
        else:
            arr[:len(dt)] = dt
        return arr

    def step(self, nsteps: int, dt):
        arr = self._dt(dt)
        _check(_lib.md_batch_step(self._h, int(nsteps), _pd(arr)))

    def step_async(self, nsteps: int, dt, stream=None):
        arr = self._dt(dt)
        _check(_lib.md_batch_step_async(self._h, int(nsteps), _pd(arr), _stream_ptr(stream)))

    def step_nvt(self, nsteps: int, dt, temperature, q, zeta=None, eta=None):
        """Nose-Hoover NVT steps of every active system (md_batch_step_nvt): dt,
        temperature and q per system (scalars, sequences or {id: value}); zeta and eta
        (max_systems arrays, zero if None) are updated and returned."""
        dts, ts, qs = self._dt(dt), self._dt(temperature), self._dt(q)
        z = np.zeros(self.max_systems) if zeta is None else np.ascontiguousarray(zeta, dtype=np.float64).copy()
        e = np.zeros(self.max_systems) if eta is None else np.ascontiguousarray(eta, dtype=np.float64).copy()
        if z.shape != (self.max_systems,) or e.shape != (self.max_systems,):
            raise ValueError(f"zeta and eta need {self.max_systems} entries")
        _check(_lib.md_batch_step_nvt(self._h, int(nsteps), _pd(dts), _pd(ts), _pd(qs), _pd(z), _pd(e)))
        return z, e

    def forces(self, sid: int) -> np.ndarray:
        f = np.empty((self._n[sid], 3))
        _check(_lib.md_batch_forces(self._h, int(sid), _pd(f)))
        return f

    def observables(self, select=None) -> np.ndarray:
        """(max_systems, 5): pe, virial, ke, T, P per id (only the ids in `select`
        when given; other rows are zero)."""
        out = np.zeros((self.max_systems, 5))
        if select is None:
            _check(_lib.md_batch_observables(self._h, _pd(out)))
        else:
            sel = np.zeros(self.max_systems, dtype=np.int32)
            sel[list(select)] = 1
            _check(_lib.md_batch_observables_select(self._h, sel.ctypes.data_as(_PI32), _pd(out)))
        return out

    def stats(self, sid: int) -> dict:
        r, s = C.c_int64(), C.c_int64()
        _check(_lib.md_batch_stats(self._h, int(sid), C.byref(r), C.byref(s)))
        return dict(rebuilds=r.value, steps=s.value)

    def kinetic_energy(self) -> np.ndarray:
        ke = np.zeros(self.max_systems)
        _check(_lib.md_batch_kinetic_energy(self._h, _pd(ke)))
        return ke

    def scale_velocities(self, factor):
        f = np.ones(self.max_systems)
        if np.isscalar(factor):
            f[:] = float(factor)
        elif isinstance(factor, dict):
            for k, val in factor.items():
                f[k] = val
        else:
            f[:len(factor)] = factor
        _check(_lib.md_batch_scale_velocities(self._h, _pd(f)))

    def set_timing(self, on: bool = True):
        _check(_lib.md_batch_set_timing(self._h, 1 if on else 0))

    def set_tuning(self, **kw):
        for k, v in kw.items():
            _check(_lib.md_batch_set_tuning(self._h, TUNING_KEYS[k], int(v)))

    def get_tuning(self) -> dict:
        out = {}
        for k, key in TUNING_KEYS.items():
            v = C.c_int()
            _check(_lib.md_batch_get_tuning(self._h, key, C.byref(v)))
            out[k] = v.value
        return out

    def get_timing(self) -> dict:
        out = np.zeros(8)
        _check(_lib.md_batch_get_timing(self._h, _pd(out)))
        return dict(step_ms=out[0], step_launches=int(out[1]), list_ms=out[2],
                    list_launches=int(out[3]), bin_ms=out[4], rebuilds=int(out[5]),
                    launches=int(out[6]))


def forces_noalloc(x, box: float, rc: float, f, stream=None):
    """md_forces_noalloc: forces of the positions in CUDA tensor x (N x 3, float64)
    into CUDA tensor f, using the library's fixed scratch array (no allocation;
    N <= 65536). Work is enqueued on stream (None = legacy default stream)."""
    n = x.numel() // 3
    _check(load_library().md_forces_noalloc(_dev_ptr(x, n), n, float(box), float(rc),
                                            _dev_ptr(f, n), _stream_ptr(stream)))


def probe_fma_rate(kind: int, iters: int) -> float:
    """md_probe_fma_rate: FMA instructions per second of the FP64 (kind 0) or FP32
    (kind 1) pipe of the current device."""
    out = C.c_double()
    _check(load_library().md_probe_fma_rate(int(kind), int(iters), C.byref(out)))
    return out.value


def version() -> str:
    return load_library().md_version().decode()

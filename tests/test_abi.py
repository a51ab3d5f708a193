"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/ljmd.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        names += re.findall(r"^MD_API\s+[\w\s\*]+?\b(md_\w+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    assert {"md_create", "md_set_state", "md_step", "md_forces", "md_observables",
            "md_destroy"} <= set(names)


def test_library_exports_every_declared_symbol(ljmd):
    lib = ctypes.CDLL(ljmd.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(ljmd):
    assert set(declared_symbols()) <= set(ljmd.SIGNATURES)


def test_version_and_error_string_without_gpu(ljmd):
    lib = ljmd.load_library()
    assert lib.md_version().decode().startswith("ljmd")
    assert isinstance(lib.md_last_error(), bytes)


def test_invalid_arguments_rejected_before_any_device_work(ljmd):
    # null output handle is rejected without touching CUDA
    lib = ljmd.load_library()
    assert lib.md_create(20.0, 10, 2.5, 0.3, None) == ljmd.MD_ERR_ARG
    assert lib.md_set_precision(None, 0) == ljmd.MD_ERR_ARG
    assert lib.md_step(None, 1, 0.005) == ljmd.MD_ERR_ARG
    lib.md_destroy(None)


def test_product_has_no_oracle_dependency():
    """The package never imports or links the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1210_3450_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\bimport oracle|from oracle|ljmd_oracle", text), f


def test_state_output_arrays_are_checked(ljmd):
    """get_state(out=...) takes caller arrays (e.g. views of pinned host memory) only
    if they are C-contiguous float64 of shape (N, 3)."""
    import numpy as np
    x, v = ljmd._out3(None, 5)
    assert x.shape == v.shape == (5, 3) and x.dtype == np.float64
    good = (np.zeros((5, 3)), np.zeros((5, 3)))
    assert ljmd._out3(good, 5)[0] is good[0]
    for bad in [(np.zeros((5, 3), np.float32), good[1]), (good[0], np.zeros((4, 3))),
                (np.zeros((3, 5)).T, good[1])]:
        with pytest.raises(ValueError):
            ljmd._out3(bad, 5)

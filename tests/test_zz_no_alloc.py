"""md_forces_noalloc, the entry point for callers that cannot let the library
allocate device memory (their device memory belongs to their own allocator or
pool, or they cannot take the synchronisation of cudaMalloc / cudaFree).

Its forces are checked against the oracle's (the all-pairs definition for small
systems, the oracle's list-based sum, itself pinned to the all-pairs sum, at the
size limit) within the FP64 force tolerance of the other tests, in every branch of
the entry point: a cell grid (two cutoffs), a box of fewer than three cells per
axis (all pairs with the minimum image), a dilute box whose cell grid is capped
at 32 per axis, and the largest size it takes, N = 65,536. Each case runs twice in
a row: the shared scratch array keeps the previous call's contents, so the second
call checks that everything that must start at zero is cleared, and the two calls
must agree bit for bit (the particles of a cell are taken in caller order, not
in the order of the atomics). One case goes through the Python binding. This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _cases():
    yield "fluid-4000", *li.perturbed_fcc(4000, 0.8442, 0.1, 201), 2.5, "brute"   # 6^3 cells
    yield "rc3-2916", *li.perturbed_fcc(2916, 0.70, 0.1, 202), 3.0, "brute"       # 5^3 cells
    yield "small-box-256", *li.perturbed_fcc(256, 0.8442, 0.1, 203), 2.5, "brute"  # L = 6.7: all pairs
    # a dense block in a mostly empty box (L / rc = 40: the grid is capped at 32
    # cells per axis), straddling a box face
    blk, _ = li.perturbed_fcc(4000, 0.8442, 0.1, 204)
    yield "dilute-box-4000", np.mod(blk + np.array([90.0, 5.0, 50.0]), 100.0), 100.0, 2.5, "brute"
    yield "max-65536", *li.perturbed_fcc(65536, 0.8442, 0.1, 205), 2.5, "list"


CASES = list(_cases())


def _call(lib, xd, fd, n, box, rc):
    r = lib.md_forces_noalloc(ctypes.c_void_p(xd.data_ptr()), n, ctypes.c_double(box), ctypes.c_double(rc),
                              ctypes.c_void_p(fd.data_ptr()), None)
    assert r == 0, lib.md_last_error()


@pytest.mark.parametrize("name,x,box,rc,ref_kind", CASES, ids=[c[0] for c in CASES])
def test_noalloc_forces_match_oracle_twice(ljmd, oracle, name, x, box, rc, ref_kind):
    import torch
    lib = ljmd.load_library()
    xw = oracle.wrap(x, box)
    ref = oracle.forces_brute(xw, box, rc) if ref_kind == "brute" else oracle.forces(xw, box, rc)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    outs = []
    for _ in range(2):
        fd = torch.full_like(xd, float("nan"))
        _call(lib, xd, fd, len(x), box, rc)
        torch.cuda.synchronize()
        outs.append(fd.cpu().numpy())
    for f in outs:
        assert np.isfinite(f).all()
        assert np.abs(f - ref).max() / rms <= FP64_TOL
    np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_through_the_binding_equals_md_forces(ljmd, oracle):
    """The Python wrapper (ljmd.forces_noalloc) on a stream, against the oracle and
    against the regular list-based md_forces at the FP64 tolerance."""
    import torch
    x, box = li.perturbed_fcc(4001, 0.8442, 0.1, 206)
    with ljmd.LJSystem(box, len(x), 2.5, 0.3) as s:
        s.set_state(x, np.zeros_like(x))
        reg = s.forces()
    ref = oracle.forces_brute(oracle.wrap(x, box), box, 2.5)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    stream = torch.cuda.Stream()
    xd = torch.from_numpy(x).cuda()
    fd = torch.empty_like(xd)
    ljmd.forces_noalloc(xd, box, 2.5, fd, stream)
    stream.synchronize()
    f = fd.cpu().numpy()
    assert np.abs(f - ref).max() / rms <= FP64_TOL
    assert np.abs(f - reg).max() / rms <= FP64_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(ljmd):
    import torch
    lib = ljmd.load_library()
    n = 65537
    xd = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    r = lib.md_forces_noalloc(ctypes.c_void_p(xd.data_ptr()), n, ctypes.c_double(50.0),
                              ctypes.c_double(2.5), ctypes.c_void_p(xd.data_ptr()), None)
    assert r == ljmd.MD_ERR_ARG
    assert b"65536" in lib.md_last_error()

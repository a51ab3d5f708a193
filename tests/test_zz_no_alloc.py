"""md_forces_noalloc, the entry point for callers that cannot let the library
allocate device memory (their device memory belongs to their own allocator, or
they cannot take the synchronisation of cudaMalloc / cudaFree). Its output must
equal the regular md_forces path within the FP64 force tolerance of the other
tests, on two calls in a row (the shared scratch array keeps the previous call's
contents, so the second call checks that everything that must start at zero is
cleared). This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _regular_forces(ljmd, x, box, rc):
    with ljmd.LJSystem(box, len(x), rc, 0.3) as s:
        s.set_state(x, np.zeros_like(x))
        return s.forces()


def test_noalloc_forces_match_regular_path_twice(ljmd):
    import torch
    lib = ljmd.load_library()
    cases = [li.perturbed_fcc(4000, 0.8442, 0.1, 201), li.perturbed_fcc(2916, 0.70, 0.1, 202)]
    for (x, box), rc in zip(cases, [2.5, 3.0]):
        ref = _regular_forces(ljmd, x, box, rc)
        xd = torch.from_numpy(x).cuda()
        fd = torch.full_like(xd, float("nan"))
        rc_ = lib.md_forces_noalloc(ctypes.c_void_p(xd.data_ptr()), len(x), ctypes.c_double(box),
                                    ctypes.c_double(rc), ctypes.c_void_p(fd.data_ptr()), None)
        assert rc_ == 0, lib.md_last_error()
        torch.cuda.synchronize()
        f = fd.cpu().numpy()
        rms = np.sqrt((ref ** 2).sum(1).mean())
        assert np.abs(f - ref).max() / rms <= FP64_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(ljmd):
    import torch
    lib = ljmd.load_library()
    n = 65537
    xd = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    rc_ = lib.md_forces_noalloc(ctypes.c_void_p(xd.data_ptr()), n, ctypes.c_double(50.0),
                                ctypes.c_double(2.5), ctypes.c_void_p(xd.data_ptr()), None)
    assert rc_ == ljmd.MD_ERR_ARG
    assert b"65536" in lib.md_last_error()

"""Nose-Hoover NVT (md_step_nvt) against the oracle's NVT integrator: positions
within 1e-9, velocities within 1e-8, thermostat variables within 1e-9 after 100
steps (only the order of the kinetic-energy sums differs), in a batch each system
equal to its run alone."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def test_nvt_matches_oracle(ljmd, oracle):
    x, box = li.perturbed_fcc(864, 0.70, 0.05, 801)
    v = li.maxwell_boltzmann(864, 1.3, 802)
    q = 0.5 * 3 * 863 * 0.9 * 0.25
    with ljmd.LJSystem(box, 864, 3.0, 0.3) as s:
        s.set_state(x, v)
        z, e = s.step_nvt(100, 0.005, 0.9, q, 0.0, 0.0)
        xg, vg = s.get_state()
    r = oracle.run_nvt(x, v, box, 3.0, 0.3, 100, 0.005, 0.9, q)
    d = xg - r["x"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(vg - r["v"]).max() < 1e-8
    assert abs(z - r["zeta"]) < 1e-9 and abs(e - r["eta"]) < 1e-9


def test_nvt_batch_equals_alone(ljmd):
    syss = li.batch_systems(count=4, seed=803)
    dt = [c.dt for c in syss]
    T = [0.9] * 4
    Q = [0.5 * 3 * (c.n - 1) * 0.9 * 0.25 for c in syss]
    import ctypes as C
    with ljmd.LJBatch(systems=[(c.n, c.box, c.rc, c.skin) for c in syss]) as b:
        for k, c in enumerate(syss):
            b.set_state(k, c.x, c.v)
        z = np.zeros(4)
        e = np.zeros(4)
        arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        dts, Ts, Qs = arr(dt), arr(T), arr(Q)
        lib = ljmd.load_library()
        pd = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        rc = lib.md_batch_step_nvt(b._h, 40, pd(dts), pd(Ts), pd(Qs), pd(z), pd(e))
        assert rc == 0, lib.md_last_error()
        for k, c in enumerate(syss):
            xb, vb = b.get_state(k)
            with ljmd.LJSystem(c.box, c.n, c.rc, c.skin) as s:
                s.set_state(c.x, c.v)
                zk, ek = s.step_nvt(40, c.dt, 0.9, Q[k])
                xs, vs = s.get_state()
            np.testing.assert_array_equal(xb, xs)
            np.testing.assert_array_equal(vb, vs)
            assert z[k] == zk and e[k] == ek

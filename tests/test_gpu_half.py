"""Half pair list with Newton's third law (each pair once, the partner's force by
atomic scatter) against the oracle.

Bars: every unordered pair within rl appears exactly once and the symmetric
closure equals the oracle's full list (integer, exact); forces within 1e-12
(FP64) and 1e-5 (FP32-force) normwise of the oracle's; PE and virial relative
1e-10; the 200-step FP64 trajectory within 1e-10 (positions) and 1e-9
(velocities) of the oracle's with the same number of list builds. The atomic
additions come in a varying order, so the graph-captured and host-driven loops,
and a system in a batch and alone, agree within 1e-9 rather than bit for bit."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def _configs():
    out = []
    x, box = li.perturbed_fcc(4000, 0.8442, 0.1, 901)
    out.append(("perturbed-4000", x, box))
    x, box = li.perturbed_fcc(4001, 0.8442, 0.1, 902)
    out.append(("perturbed-4001", x, box))
    x, box = li.perturbed_fcc(518, 0.8442, 0.1, 903)
    out.append(("three-cells-518", x, box))
    x, box = li.perturbed_fcc(300, 0.85, 0.1, 904)
    out.append(("small-box-300", x, box))
    x, box = li.perturbed_fcc(33, 0.1, 0.2, 905)
    out.append(("dilute-33", x, box))
    return out


CONFIGS = _configs()
IDS = [c[0] for c in CONFIGS]


def force_err(f, ref):
    rms = np.sqrt((ref ** 2).sum(1).mean())
    return np.abs(f - ref).max() / rms


def half(ljmd, x, v, box, precision=0):
    s = ljmd.LJSystem(box, len(x), 2.5, 0.3, precision)
    s.set_pair_list(ljmd.MD_LIST_HALF)
    s.set_state(x, v)
    return s


@pytest.mark.parametrize("name,x,box", CONFIGS, ids=IDS)
def test_half_list_holds_each_pair_once(ljmd, oracle, name, x, box):
    with half(ljmd, x, np.zeros_like(x), box) as s:
        start, partners = s.get_list()
    n = len(x)
    i = np.repeat(np.arange(n), np.diff(start))
    j = partners.astype(np.int64)
    a, b = np.minimum(i, j), np.maximum(i, j)
    key = a * n + b
    assert len(np.unique(key)) == len(key)              # no pair twice
    ostart, opartners = oracle.build_list(oracle.wrap(x, box), box, 2.8)
    assert len(key) * 2 == ostart[-1]
    # symmetric closure, sorted per particle, equals the full list
    ii = np.concatenate([i, j])
    jj = np.concatenate([j, i])
    order = np.lexsort((jj, ii))
    np.testing.assert_array_equal(np.bincount(ii, minlength=n), np.diff(ostart))
    np.testing.assert_array_equal(jj[order], opartners)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,x,box", CONFIGS, ids=IDS)
def test_half_list_forces(ljmd, oracle, name, x, box, precision, tol):
    with half(ljmd, x, np.zeros_like(x), box, precision) as s:
        f = s.forces()
    xw = oracle.wrap(x, box)
    assert force_err(f, oracle.forces(xw, box, 2.5)) <= tol
    assert force_err(f, oracle.forces_half(xw, box, 2.5)) <= tol


def test_half_list_observables(ljmd, oracle):
    x, box = li.perturbed_fcc(4000, 0.8442, 0.1, 906)
    v = li.maxwell_boltzmann(4000, 0.722, 907)
    with half(ljmd, x, v, box) as s:
        o = s.observables()
    ro = oracle.observables(oracle.wrap(x, box), v, box, 2.5)
    assert o["pe"] == pytest.approx(ro["pe"], rel=1e-10)
    assert o["virial"] == pytest.approx(ro["virial"], rel=1e-10)


def test_half_list_trajectory_fp64(ljmd, oracle):
    cfg = li.config_small_fluid()
    with half(ljmd, cfg.x, cfg.v, cfg.box) as s:
        s.step(cfg.steps, cfg.dt)
        xg, vg = s.get_state()
        st = s.stats()
    r = oracle.run(cfg.x, cfg.v, cfg.box, cfg.rc, cfg.skin, cfg.steps, cfg.dt)
    d = xg - r["x"]
    d -= cfg.box * np.round(d / cfg.box)
    assert np.abs(d).max() < 1e-10
    assert np.abs(vg - r["v"]).max() < 1e-9
    assert st["rebuilds"] == r["rebuilds"]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_half_list_graph_and_batch(ljmd, precision):
    x, box = li.perturbed_fcc(3000, 0.8442, 0.08, 908)
    v = li.maxwell_boltzmann(3000, 1.0, 909)
    out = []
    for graph in (0, 1):
        with half(ljmd, x, v, box, precision) as s:
            s.set_tuning(graph=graph)
            s.step(101, 0.005)
            out.append(s.get_state())
    x2, box2 = li.perturbed_fcc(1200, 0.7, 0.08, 910)
    v2 = li.maxwell_boltzmann(1200, 1.0, 911)
    b = ljmd.LJBatch(systems=[(3000, box, 2.5, 0.3), (1200, box2, 2.5, 0.3)], precision=precision)
    try:
        b.set_pair_list(ljmd.MD_LIST_HALF)
        b.set_state(0, x, v)
        b.set_state(1, x2, v2)
        b.step(101, [0.005, 0.005])
        out.append(b.get_state(0))
    finally:
        b.close()
    for xs, vs in out[1:]:
        assert np.abs(xs - out[0][0]).max() < 1e-9
        assert np.abs(vs - out[0][1]).max() < 1e-8


def test_switching_list_form_keeps_forces(ljmd):
    x, box = li.perturbed_fcc(4000, 0.8442, 0.1, 912)
    with ljmd.LJSystem(box, 4000, 2.5, 0.3) as s:
        s.set_state(x, np.zeros_like(x))
        f_full = s.forces()
        s.set_pair_list(ljmd.MD_LIST_HALF)
        f_half = s.forces()
        s.set_pair_list(ljmd.MD_LIST_FULL)
        f_back = s.forces()
    assert force_err(f_half, f_full) < 1e-13
    np.testing.assert_array_equal(f_back, f_full)

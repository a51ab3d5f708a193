"""List validity by the velocity bound (the DUTC check of Sec. 2.1) on the GPU.

Bars: the FP64 trajectory of the 4000-particle fluid under the velocity bound
matches the oracle's (same rule) within 1e-10 in positions and 1e-9 in
velocities, with the same number of list builds; a vibrating dimer rebuilds
exactly as often as in the oracle under either rule; the graph-captured loop
equals the host-driven one bit for bit, and a batched system equals its run
alone, under the velocity bound."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def test_dutc_trajectory_matches_oracle(ljmd, oracle):
    cfg = li.config_small_fluid()
    v = li.maxwell_boltzmann(cfg.n, 1.1, 801)
    with ljmd.LJSystem(cfg.box, cfg.n, cfg.rc, cfg.skin, ljmd.MD_FP64) as s:
        s.set_validity_rule(ljmd.MD_RULE_DUTC)
        s.set_state(cfg.x, v)
        s.step(cfg.steps, cfg.dt)
        xg, vg = s.get_state()
        st = s.stats()
    r = oracle.run(cfg.x, v, cfg.box, cfg.rc, cfg.skin, cfg.steps, cfg.dt, rule=1)
    d = xg - r["x"]
    d -= cfg.box * np.round(d / cfg.box)
    assert np.abs(d).max() < 1e-10
    assert np.abs(vg - r["v"]).max() < 1e-9
    assert st["rebuilds"] == r["rebuilds"] > 10


@pytest.mark.parametrize("rule", [0, 1], ids=["displacement", "dutc"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_vibrating_dimer_rebuild_count(ljmd, oracle, rule, precision):
    x = np.array([[5.0, 5.0, 5.0], [6.2, 5.0, 5.0]])
    v = np.zeros((2, 3))
    with ljmd.LJSystem(12.0, 2, 2.5, 0.3, precision) as s:
        s.set_validity_rule(rule)
        s.set_state(x, v)
        s.step(2000, 0.005)
        st = s.stats()
    r = oracle.run(x, v, 12.0, 2.5, 0.3, 2000, 0.005, rule=rule)
    assert st["rebuilds"] == r["rebuilds"]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_dutc_graph_equals_host_loop(ljmd, precision):
    x, box = li.perturbed_fcc(3000, 0.8442, 0.08, 802)
    v = li.maxwell_boltzmann(3000, 1.1, 803)
    out = []
    for graph in (0, 1):
        with ljmd.LJSystem(box, 3000, 2.5, 0.3, precision) as s:
            s.set_tuning(graph=graph)
            s.set_validity_rule(ljmd.MD_RULE_DUTC)
            s.set_state(x, v)
            s.step(151, 0.005)
            out.append(s.get_state() + (s.stats(),))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_dutc_batch_equals_alone(ljmd):
    specs, states = [], []
    for n, rho, seed in [(1500, 0.8, 804), (4000, 0.7, 805), (400, 0.85, 806)]:
        x, box = li.perturbed_fcc(n, rho, 0.08, seed)
        specs.append((n, box, 2.5, 0.3))
        states.append((x, li.maxwell_boltzmann(n, 1.0, seed + 100)))
    b = ljmd.LJBatch(systems=specs, precision=ljmd.MD_FP32_FORCE)
    try:
        b.set_validity_rule(ljmd.MD_RULE_DUTC)
        for k, (x, v) in enumerate(states):
            b.set_state(k, x, v)
        b.step(120, [0.005] * len(specs))
        got = [b.get_state(k) + (b.stats(k),) for k in range(len(specs))]
    finally:
        b.close()
    for (n, box, rc, skin), (x, v), (xb, vb, sb) in zip(specs, states, got):
        with ljmd.LJSystem(box, n, rc, skin, ljmd.MD_FP32_FORCE) as s:
            s.set_validity_rule(ljmd.MD_RULE_DUTC)
            s.set_state(x, v)
            s.step(120, 0.005)
            xa, va = s.get_state()
            sa = s.stats()
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(va, vb)
        assert sa == sb

"""Checkpoint and resume: a run stopped at any step, checkpointed (positions as
held, velocities, positions at the last list build, velocity-bound margin) and
restored into a new context continues exactly as the uninterrupted run, bit for
bit, under both list validity rules and in both force forms."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rule", [0, 1], ids=["displacement", "dutc"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_resume_equals_uninterrupted(ljmd, precision, rule):
    x, box = li.perturbed_fcc(4000, 0.8442, 0.08, 1101)
    v = li.maxwell_boltzmann(4000, 1.1, 1102)

    def fresh():
        s = ljmd.LJSystem(box, 4000, 2.5, 0.3, precision)
        s.set_validity_rule(rule)
        return s

    with fresh() as a:
        a.set_state(x, v)
        a.step(300, 0.005)
        xa, va = a.get_state()
    with fresh() as b:
        b.set_state(x, v)
        b.step(131, 0.005)
        done = 131
        ck = b.checkpoint()
        while np.all(ck["x"] == ck["x_build"]):     # stop between list builds
            b.step(1, 0.005)
            done += 1
            ck = b.checkpoint()
    with fresh() as c:
        c.restore(ck)
        c.step(300 - done, 0.005)
        xc, vc = c.get_state()
    np.testing.assert_array_equal(xa, xc)
    np.testing.assert_array_equal(va, vc)


def test_checkpoint_right_after_set_state(ljmd):
    x, box = li.perturbed_fcc(1000, 0.8, 0.1, 1103)
    v = li.maxwell_boltzmann(1000, 1.0, 1104)
    with ljmd.LJSystem(box, 1000, 2.5, 0.3) as s:
        s.set_state(x, v)
        ck = s.checkpoint()
        np.testing.assert_array_equal(ck["x_build"], ck["x"])
        np.testing.assert_array_equal(ck["v"], v)
        assert ck["margin"] == 0.3
    with ljmd.LJSystem(box, 1000, 2.5, 0.3) as s:
        with pytest.raises(ljmd.MDError) as e:
            s.checkpoint()
        assert e.value.code == ljmd.MD_ERR_STATE


def test_batch_checkpoint_moves_a_system(ljmd):
    """A system of a batch checkpointed mid-run and resumed in another batch (beside
    systems at other points of their runs) and in a single context continues bit for
    bit as the uninterrupted run: the eviction and resumption a server does."""
    specs, states = [], []
    for n, rho, seed in [(1200, 0.8, 1111), (3000, 0.75, 1113), (800, 0.85, 1115)]:
        x, box = li.perturbed_fcc(n, rho, 0.08, seed)
        specs.append((n, box, 2.5, 0.3))
        states.append((x, li.maxwell_boltzmann(n, 1.0, seed + 1)))
    dts = [0.005, 0.004, 0.005]

    def batch():
        b = ljmd.LJBatch(systems=specs, precision=ljmd.MD_FP32_FORCE)
        for k, (x, v) in enumerate(states):
            b.set_state(k, x, v)
        return b

    a = batch()
    try:
        a.step(97, dts)
        ck = a.checkpoint(1)
        a.step(60, dts)
        ref = a.get_state(1)
    finally:
        a.close()
    c = batch()
    try:
        c.step(13, dts)                     # the others are elsewhere in their runs
        c.restore(1, ck)
        c.step(60, dts)
        got = c.get_state(1)
    finally:
        c.close()
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    n, box = specs[1][0], specs[1][1]
    with ljmd.LJSystem(box, n, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(*states[1])
        s.restore(ck)
        s.step(60, 0.004)
        alone = s.get_state()
    np.testing.assert_array_equal(alone[0], ref[0])
    np.testing.assert_array_equal(alone[1], ref[1])

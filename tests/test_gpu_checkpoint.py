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

"""Launch shapes change speed only: results are bit-for-bit the same for every
tuning, and the autotuner picks one of the allowed shapes."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_tuning_does_not_change_results(ljmd, precision):
    x, box = li.perturbed_fcc(3000, 0.8442, 0.08, 501)
    v = li.maxwell_boltzmann(3000, 0.9, 502)
    outs = []
    for tun in [dict(step_block=128, step_groups=1, list_block=128, list_variant=5, step_hint=0),
                dict(step_block=64, step_groups=2, list_block=256, list_variant=3, step_hint=1),
                dict(step_block=256, step_groups=2, list_block=64, list_variant=4, step_hint=1),
                dict(step_block=128, step_groups=1, list_block=128, list_variant=2, step_hint=1),
                dict(step_block=128, step_groups=2, list_block=256, list_variant=1, step_hint=1,
                     fp64_queue=0)]:
        with ljmd.LJSystem(box, 3000, 2.5, 0.3, precision) as s:
            s.set_tuning(**tun)
            got = s.get_tuning()
            assert {k: got[k] for k in tun} == tun
            s.set_state(x, v)
            s.step(60, 0.005)
            outs.append(s.get_state())
    for x1, v1 in outs[1:]:
        np.testing.assert_array_equal(x1, outs[0][0])
        np.testing.assert_array_equal(v1, outs[0][1])


def test_autotuner_picks_valid_shape(ljmd, tmp_path):
    from paper_1210_3450_gb300 import autotune
    x, box = li.perturbed_fcc(4000, 0.8442, 0.08, 503)
    with ljmd.LJSystem(box, 4000, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, li.maxwell_boltzmann(4000, 0.722, 504))
        cache = str(tmp_path / "tune.json")
        res = autotune.tune(s, 0.005, key="t", steps=10, cache=cache)
        t = s.get_tuning()
        assert t == res["tuning"]
        assert t["step_block"] in autotune.STEP_BLOCKS and t["step_groups"] in autotune.STEP_GROUPS
        assert t["step_hint"] in autotune.STEP_HINTS
        again = autotune.tune(s, 0.005, key="t", cache=cache)   # from the cache, no timing
        assert again["tuning"] == res["tuning"]
    with pytest.raises(ljmd.MDError):
        with ljmd.LJSystem(box, 4000, 2.5, 0.3) as s:
            s.set_tuning(step_block=100)

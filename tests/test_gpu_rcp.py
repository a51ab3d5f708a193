"""The paper's FX10 force kernel variant (Sec. 3.3): r^-8 and r^-14 from an
approximate reciprocal of r^2, with and without the correction of Eqs. 2-7.

Bars: forces of each variant equal the oracle's implementation of the same
variant (same approximate reciprocal, FP64 polynomial) within 1e-12 normwise;
and, as in Fig. 3 (N = 4000, energy of a run with and without the correction),
the corrected 8-bit form conserves energy better than the uncorrected one, and
the corrected 23-bit form as well as exact FP64 (within 2x)."""
import json

import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu

MODES = {2: (8, False), 3: (8, True), 4: (23, False), 5: (23, True)}


@pytest.mark.parametrize("mode", sorted(MODES))
def test_rcp_forces_match_oracle_variant(ljmd, oracle, mode):
    bits, corr = MODES[mode]
    x, box = li.perturbed_fcc(4000, 0.8442, 0.1, 601)
    with ljmd.LJSystem(box, 4000, 2.5, 0.3, mode) as s:
        s.set_state(x, np.zeros_like(x))
        f = s.forces()
    ref = oracle.forces_rcp(x, box, 2.5, bits, corr)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert np.abs(f - ref).max() / rms <= 1e-12


def test_correction_improves_energy_conservation(ljmd):
    x, box = li.perturbed_fcc(4000, 0.8442, 0.05, 602)
    v = li.maxwell_boltzmann(4000, 0.722, 603)
    drift = {}
    for mode in [0, 2, 3, 4, 5]:
        e = []
        with ljmd.LJSystem(box, 4000, 2.5, 0.3, mode) as s:
            s.set_state(x, v)
            o = s.observables()
            e.append(o["pe"] + o["ke"])
            for _ in range(20):
                s.step(100, 0.005)
                o = s.observables()
                e.append(o["pe"] + o["ke"])
        e = np.array(e)
        drift[mode] = float(np.abs(e - e[0]).max() / 4000)
    print(json.dumps({"drift_per_particle": drift}))
    assert drift[2] > 2.0 * drift[3]
    assert drift[5] <= 2.0 * drift[0]

"""FP32-force form against the FP64 oracle: energy drift over 10^4 steps and the
error of each observable.

Bars: the N = 4000 fluid (rho 0.8442, T 0.722, dt 0.005): the FP32-force drift
max_t |E(t) - E(0)| / N over 10^4 steps is at most twice the oracle's (E = KE + PE,
sampled every 100 steps); after one step |dPE| / N, |dW| / N and |dT| against the
oracle are below 1e-7, 1e-6 and 1e-8. Later differences are reported, not gated
(trajectories decorrelate: the dynamics is chaotic).
"""
import json

import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def _gpu_trace(ljmd, cfg, precision, nsteps, every):
    trace = []
    with ljmd.LJSystem(cfg.box, cfg.n, cfg.rc, cfg.skin, precision) as s:
        s.set_state(cfg.x, cfg.v)
        o = s.observables()
        trace.append(o["pe"] + o["ke"])
        for _ in range(nsteps // every):
            s.step(every, cfg.dt)
            o = s.observables()
            trace.append(o["pe"] + o["ke"])
    return np.array(trace)


def test_energy_drift_fp32_within_twice_oracle(ljmd, oracle):
    cfg = li.config_small_fluid()
    nsteps, every = 10_000, 100
    ref = oracle.run(cfg.x, cfg.v, cfg.box, cfg.rc, cfg.skin, nsteps, cfg.dt, trace_every=every)["trace"]
    e32 = _gpu_trace(ljmd, cfg, 1, nsteps, every)
    e64 = _gpu_trace(ljmd, cfg, 0, nsteps, every)
    d_ref = np.abs(ref - ref[0]).max() / cfg.n
    d32 = np.abs(e32 - e32[0]).max() / cfg.n
    d64 = np.abs(e64 - e64[0]).max() / cfg.n
    print(json.dumps(dict(drift_oracle=d_ref, drift_fp32=d32, drift_fp64=d64)))
    assert d32 <= 2.0 * d_ref
    assert d64 <= 2.0 * d_ref


def test_observable_errors_fp32(ljmd, oracle):
    cfg = li.config_small_fluid()
    x, box = li.perturbed_fcc(cfg.n, 0.8442, 0.1, 401)     # nonzero forces from step 0
    v = li.maxwell_boltzmann(cfg.n, 0.722, 402)
    report = {}
    for nsteps in (1, 200):
        r = oracle.run(x, v, box, cfg.rc, cfg.skin, nsteps, cfg.dt)
        ro = oracle.observables(r["x"], r["v"], box, cfg.rc)
        with ljmd.LJSystem(box, cfg.n, cfg.rc, cfg.skin, 1) as s:
            s.set_state(x, v)
            s.step(nsteps, cfg.dt)
            o = s.observables()
        report[nsteps] = dict(dpe_per_n=abs(o["pe"] - ro["pe"]) / cfg.n,
                              dw_per_n=abs(o["virial"] - ro["virial"]) / cfg.n,
                              dT=abs(o["temperature"] - ro["temperature"]))
    print(json.dumps(report))
    assert report[1]["dpe_per_n"] < 1e-7
    assert report[1]["dw_per_n"] < 1e-6
    assert report[1]["dT"] < 1e-8

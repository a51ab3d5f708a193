"""Batched replicas and the continuous-batching arena (md_batch_*).

Bar: every system's state, rebuild count and observables after a batched run are
bit-for-bit those of the same system run alone (the kernels do no cross-system
arithmetic and every per-system reduction has a fixed order), in both precision
modes; systems added to and removed from a running arena keep that property.
"""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def _systems():
    out = []
    x, box = li.perturbed_fcc(4000, 0.8442, 0.08, 301)
    out.append(dict(x=x, v=li.maxwell_boltzmann(4000, 0.722, 302), box=box, rc=2.5, skin=0.3, dt=0.005))
    x, box = li.perturbed_fcc(500, 0.85, 0.05, 303)          # fewer than 3 cells: all pairs
    out.append(dict(x=x, v=li.maxwell_boltzmann(500, 1.2, 304), box=box, rc=2.5, skin=0.3, dt=0.004))
    x, box = li.perturbed_fcc(1999, 0.60, 0.1, 305)          # ragged tile
    out.append(dict(x=x, v=li.maxwell_boltzmann(1999, 1.0, 306), box=box, rc=2.5, skin=0.3, dt=0.005))
    x, box = li.perturbed_fcc(2916, 0.70, 0.1, 307)           # rc = 3.0
    out.append(dict(x=x, v=li.maxwell_boltzmann(2916, 0.9, 308), box=box, rc=3.0, skin=0.3, dt=0.005))
    x, box = li.perturbed_fcc(33, 0.1, 0.2, 309)
    out.append(dict(x=x, v=li.maxwell_boltzmann(33, 0.8, 310), box=box, rc=2.5, skin=0.3, dt=0.003))
    return out


def _alone(ljmd, s, nsteps, precision):
    with ljmd.LJSystem(s["box"], len(s["x"]), s["rc"], s["skin"], precision) as m:
        m.set_state(s["x"], s["v"])
        m.step(nsteps, s["dt"])
        x, v = m.get_state()
        return x, v, m.stats()["rebuilds"], m.observables()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_batch_equals_alone_bitwise(ljmd, precision):
    syss = _systems()
    nsteps = 60
    ref = [_alone(ljmd, s, nsteps, precision) for s in syss]
    with ljmd.LJBatch(systems=[(len(s["x"]), s["box"], s["rc"], s["skin"]) for s in syss],
                      precision=precision) as b:
        for k, s in enumerate(syss):
            b.set_state(k, s["x"], s["v"])
        b.step(nsteps, [s["dt"] for s in syss])
        obs = b.observables()
        for k in range(len(syss)):
            x, v = b.get_state(k)
            np.testing.assert_array_equal(x, ref[k][0])
            np.testing.assert_array_equal(v, ref[k][1])
            assert b.stats(k)["rebuilds"] == ref[k][2]
            o = ref[k][3]
            np.testing.assert_array_equal(obs[k], [o["pe"], o["virial"], o["ke"], o["temperature"], o["pressure"]])


def test_batch_forces_match_oracle(ljmd, oracle):
    syss = _systems()
    with ljmd.LJBatch(systems=[(len(s["x"]), s["box"], s["rc"], s["skin"]) for s in syss]) as b:
        for k, s in enumerate(syss):
            b.set_state(k, s["x"], s["v"])
        for k, s in enumerate(syss):
            f = b.forces(k)
            ref = oracle.forces_brute(s["x"], s["box"], s["rc"])
            rms = np.sqrt((ref ** 2).sum(1).mean())
            assert np.abs(f - ref).max() / rms <= 1e-12


def test_batch_fp32_forces_match_oracle(ljmd, oracle):
    """FP32-force form in a batch: each system's forces within the FP32 bar (max
    |F - F_ref| / rms F_ref <= 1e-5) of the oracle's all-pairs sum."""
    syss = _systems()
    with ljmd.LJBatch(systems=[(len(s["x"]), s["box"], s["rc"], s["skin"]) for s in syss],
                      precision=ljmd.MD_FP32_FORCE) as b:
        for k, s in enumerate(syss):
            b.set_state(k, s["x"], s["v"])
        for k, s in enumerate(syss):
            f = b.forces(k)
            ref = oracle.forces_brute(s["x"], s["box"], s["rc"])
            rms = np.sqrt((ref ** 2).sum(1).mean())
            assert np.abs(f - ref).max() / rms <= 1e-5


@pytest.mark.parametrize("graph", [0, 1], ids=["host", "graph"])
def test_system_order_does_not_change_results(ljmd, graph):
    """Rebuild passes take the systems in descending estimated list-build cost,
    ties by system index; that order only schedules work. The same systems placed
    in the arena forward and reversed (two of them with equal cost, so the tie
    order differs) end bit for bit alike."""
    syss = _systems()
    twin = dict(syss[0])
    twin["v"] = li.maxwell_boltzmann(4000, 0.9, 311)   # same size and box, other velocities
    syss.append(twin)
    runs = []
    for order in (list(range(len(syss))), list(reversed(range(len(syss))))):
        with ljmd.LJBatch(systems=[(len(syss[i]["x"]), syss[i]["box"], syss[i]["rc"], syss[i]["skin"])
                                   for i in order], precision=ljmd.MD_FP32_FORCE) as b:
            b.set_tuning(graph=graph)
            for k, i in enumerate(order):
                b.set_state(k, syss[i]["x"], syss[i]["v"])
            b.step(120, [syss[i]["dt"] for i in order])
            got = {}
            for k, i in enumerate(order):
                x, v = b.get_state(k)
                got[i] = (x, v, b.stats(k)["rebuilds"])
            runs.append(got)
    for i in range(len(syss)):
        np.testing.assert_array_equal(runs[0][i][0], runs[1][i][0])
        np.testing.assert_array_equal(runs[0][i][1], runs[1][i][1])
        assert runs[0][i][2] == runs[1][i][2]


def test_arena_add_remove_keeps_results(ljmd):
    """Continuous batching: B runs throughout; A leaves after 30 steps and C takes
    its place; B and C end bit-for-bit equal to their runs alone."""
    syss = _systems()
    A, B, C = syss[0], syss[2], syss[3]
    fps = [ljmd.footprint(len(s["x"]), s["box"], s["rc"], s["skin"]) for s in (A, B, C)]
    arena = dict(slots=sum(f["slots"] for f in fps[:2]) + 64,
                 cells=sum(f["cells"] for f in fps) + 16,
                 list_words=sum(f["list_words"] for f in fps[:2]) + fps[2]["list_words"] + 4096,
                 max_systems=4)
    for precision in (0, 1):
        with ljmd.LJBatch(arena=arena, precision=precision) as b:
            ia = b.add(len(A["x"]), A["box"], A["rc"], A["skin"])
            ib = b.add(len(B["x"]), B["box"], B["rc"], B["skin"])
            b.set_state(ia, A["x"], A["v"])
            b.set_state(ib, B["x"], B["v"])
            b.step(30, {ia: A["dt"], ib: B["dt"]})
            # C does not fit while A is there
            assert b.try_add(len(C["x"]), C["box"], C["rc"], C["skin"]) is None
            b.remove(ia)
            ic = b.add(len(C["x"]), C["box"], C["rc"], C["skin"])
            b.set_state(ic, C["x"], C["v"])
            b.step(30, {ib: B["dt"], ic: C["dt"]})
            xb, vb = b.get_state(ib)
            xc, vc = b.get_state(ic)
            u = b.usage()
            assert u["systems_used"] == 2
        rb = _alone(ljmd, B, 60, precision)
        rc_ = _alone(ljmd, C, 30, precision)
        np.testing.assert_array_equal(xb, rb[0])
        np.testing.assert_array_equal(vb, rb[1])
        np.testing.assert_array_equal(xc, rc_[0])
        np.testing.assert_array_equal(vc, rc_[1])


def test_inactive_system_is_frozen(ljmd):
    syss = _systems()[:2]
    with ljmd.LJBatch(systems=[(len(s["x"]), s["box"], s["rc"], s["skin"]) for s in syss]) as b:
        for k, s in enumerate(syss):
            b.set_state(k, s["x"], s["v"])
        x0, v0 = b.get_state(1)
        b.set_active(1, False)
        b.step(10, [s["dt"] for s in syss])
        x1, v1 = b.get_state(1)
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(v0, v1)
        assert b.stats(0)["steps"] == 10 and b.stats(1)["steps"] == 0


def test_replica_workload_sample_matches_alone(ljmd):
    """32 systems drawn like the 256-replica workload (N log-uniform in
    [500, 32000], rho in [0.60, 0.85], T in [0.7, 1.2]) in FP32-force mode:
    each equals its run alone after 40 steps."""
    syss = li.batch_systems(count=32, seed=1004)
    with ljmd.LJBatch(systems=[(c.n, c.box, c.rc, c.skin) for c in syss], precision=1) as b:
        for k, c in enumerate(syss):
            b.set_state(k, c.x, c.v)
        b.step(40, [c.dt for c in syss])
        for k in [0, 7, 13, 31]:
            c = syss[k]
            x, v = b.get_state(k)
            with ljmd.LJSystem(c.box, c.n, c.rc, c.skin, 1) as m:
                m.set_state(c.x, c.v)
                m.step(40, c.dt)
                xr, vr = m.get_state()
            np.testing.assert_array_equal(x, xr)
            np.testing.assert_array_equal(v, vr)


@pytest.mark.parametrize("graph", [0, 1], ids=["host-loop", "graph"])
def test_paused_system_resumes_exactly(ljmd, graph):
    """A system set inactive while the others advance an odd number of steps (the
    position buffers alternate by step) resumes from its own positions: its run
    equals the run alone bit for bit."""
    import lj_inputs as li
    x1, b1 = li.perturbed_fcc(2000, 0.8, 0.08, 1201)
    v1 = li.maxwell_boltzmann(2000, 1.0, 1202)
    x2, b2 = li.perturbed_fcc(1500, 0.75, 0.08, 1203)
    v2 = li.maxwell_boltzmann(1500, 1.0, 1204)
    b = ljmd.LJBatch(systems=[(2000, b1, 2.5, 0.3), (1500, b2, 2.5, 0.3)], precision=ljmd.MD_FP32_FORCE)
    try:
        b.set_tuning(graph=graph)
        b.set_state(0, x1, v1)
        b.set_state(1, x2, v2)
        b.step(20, [0.005, 0.005])
        b.set_active(1, False)
        b.step(7, [0.005, 0.005])          # system 0 only, odd count
        b.set_active(1, True)
        b.step(33, [0.005, 0.005])
        xb, vb = b.get_state(1)
    finally:
        b.close()
    with ljmd.LJSystem(b2, 1500, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x2, v2)
        s.step(53, 0.005)
        xa, va = s.get_state()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)


def test_empty_and_paused_arena_steps_are_no_ops(ljmd):
    """Stepping an arena with no systems, or with every system paused, does nothing
    and succeeds; a system added afterwards steps as it does alone."""
    x, box = li.perturbed_fcc(700, 0.8, 0.1, 631)
    v = li.maxwell_boltzmann(700, 0.9, 632)
    b = ljmd.LJBatch(arena=dict(slots=4096, cells=4096, list_words=1 << 20, max_systems=4),
                     precision=ljmd.MD_FP32_FORCE)
    try:
        b.step(5, [0.005] * b.max_systems)
        b.step_nvt(4, [0.005] * b.max_systems, [1.0] * b.max_systems, [1.0] * b.max_systems)
        sid = b.add(700, box, 2.5, 0.3)
        b.set_state(sid, x, v)
        before = b.get_state(sid)
        b.set_active(sid, False)
        b.step(5, [0.005] * b.max_systems)
        b.set_active(sid, True)
        after = b.get_state(sid)
        np.testing.assert_array_equal(after[0], before[0])
        np.testing.assert_array_equal(after[1], before[1])
        b.step(20, [0.005] * b.max_systems)
        got = b.get_state(sid)
        b.remove(sid)
        b.step(3, [0.005] * b.max_systems)
    finally:
        b.close()
    with ljmd.LJSystem(box, 700, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, v)
        s.step(20, 0.005)
        ref = s.get_state()
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])


def test_device_state_calls_match_host_calls(ljmd):
    """set_state_dev / get_state_dev (CUDA tensors, caller order) give the same
    state as the host-array calls, for one system and for a system of a batch."""
    import torch
    x, box = li.perturbed_fcc(1500, 0.8, 0.1, 641)
    v = li.maxwell_boltzmann(1500, 0.9, 642)
    xd = torch.tensor(x, device="cuda")
    vd = torch.tensor(v, device="cuda")
    with ljmd.LJSystem(box, 1500, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state_dev(xd, vd)
        s.step(30, 0.005)
        xo, vo = torch.empty_like(xd), torch.empty_like(vd)
        s.get_state_dev(xo, vo)
        torch.cuda.synchronize()
        xh, vh = s.get_state()
    np.testing.assert_array_equal(xo.cpu().numpy(), xh)
    np.testing.assert_array_equal(vo.cpu().numpy(), vh)
    b = ljmd.LJBatch(systems=[(700, li.box_length(700, 0.8), 2.5, 0.3), (1500, box, 2.5, 0.3)],
                     precision=ljmd.MD_FP32_FORCE)
    try:
        x0, b0 = li.perturbed_fcc(700, 0.8, 0.1, 643)
        b.set_state(0, x0, li.maxwell_boltzmann(700, 0.9, 644))
        b.set_state_dev(1, xd, vd)
        b.step(30, [0.005, 0.005])
        xo2, vo2 = torch.empty_like(xd), torch.empty_like(vd)
        b.get_state_dev(1, xo2, vo2)
        torch.cuda.synchronize()
        xb, vb = b.get_state(1)
    finally:
        b.close()
    np.testing.assert_array_equal(xo2.cpu().numpy(), xb)
    np.testing.assert_array_equal(vo2.cpu().numpy(), vb)
    np.testing.assert_array_equal(xb, xh)   # the same system, alone and in a batch
    np.testing.assert_array_equal(vb, vh)

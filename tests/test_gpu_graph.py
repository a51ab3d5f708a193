"""The graph-captured step loop (a CUDA graph per chunk of steps: loop node,
device-side list-validity decision, conditional rebuild) against the
host-driven loop (the host decides after every step).

Bars: positions, velocities and rebuild counts bit for bit equal, for one
system in the FP32-force and FP64 forms, for a batch of uneven systems
(including one small enough that every pair is a candidate), across an odd
step count (the last step runs host-driven), and through a list overflow in a
rebuild inside the graph (the host grows the list and resumes); a non-finite
value stops the loop with the same error."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def run(ljmd, x, v, box, precision, graph, steps, tuning=None):
    with ljmd.LJSystem(box, len(x), 2.5, 0.3, precision) as s:
        s.set_tuning(graph=graph, **(tuning or {}))
        assert s.get_tuning()["graph"] == graph
        s.set_state(x, v)
        s.step(steps, 0.005)
        s.step(steps // 3, 0.005)          # a second call continues the same run
        xs, vs = s.get_state()
        return xs, vs, s.stats()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_single_system_equals_host_loop(ljmd, precision):
    x, box = li.perturbed_fcc(4000, 0.8442, 0.08, 701)
    v = li.maxwell_boltzmann(4000, 1.1, 702)
    a = run(ljmd, x, v, box, precision, 0, 201)
    b = run(ljmd, x, v, box, precision, 1, 201)
    assert a[2]["rebuilds"] > 10
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2]


def test_warp_list_variant_in_graph(ljmd):
    x, box = li.perturbed_fcc(3000, 0.8442, 0.08, 703)
    v = li.maxwell_boltzmann(3000, 1.1, 704)
    a = run(ljmd, x, v, box, 1, 0, 120)
    b = run(ljmd, x, v, box, 1, 1, 120, tuning=dict(list_variant=4))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_batch_equals_host_loop(ljmd):
    rng = np.random.default_rng(705)
    specs, states = [], []
    for n, rho in [(300, 0.85), (2000, 0.8), (5000, 0.7), (900, 0.6), (7000, 0.82)]:
        x, box = li.perturbed_fcc(n, rho, 0.08, int(rng.integers(1 << 30)))
        v = li.maxwell_boltzmann(n, float(rng.uniform(0.8, 1.2)), int(rng.integers(1 << 30)))
        specs.append((n, box, 2.5, 0.3))
        states.append((x, v))
    dts = [0.005, 0.004, 0.005, 0.003, 0.005]
    out = []
    for graph in (0, 1):
        b = ljmd.LJBatch(systems=specs, precision=ljmd.MD_FP32_FORCE)
        try:
            b.set_tuning(graph=graph)
            for k, (x, v) in enumerate(states):
                b.set_state(k, x, v)
            b.step(150, dts)
            b.step(7, dts)
            out.append([b.get_state(k) + (b.stats(k),) for k in range(len(specs))])
        finally:
            b.close()
    for (x0, v0, s0), (x1, v1, s1) in zip(*out):
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(v0, v1)
        assert s0 == s1


def test_overflow_inside_graph_grows_and_resumes(ljmd, oracle):
    """A dilute lattice gas contracting towards the centre: the density rises
    about eightfold, so a rebuild inside the graph overflows the initial list
    capacity."""
    n = 1372
    x, box = li.perturbed_fcc(n, 0.0556, 0.1, 706)   # lattice: no close pairs to blow up
    v = -0.38 * (x - 0.5 * box)
    rl = 2.8
    kmax0 = -(-int(1.35 * 4.0 / 3.0 * np.pi * rl ** 3 * n / box ** 3 + 32.0) // 8) * 8
    res = []
    for graph in (0, 1):
        with ljmd.LJSystem(box, n, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
            s.set_tuning(graph=graph)
            s.set_state(x, v)
            s.step(300, 0.005)
            xs, vs = s.get_state()
            st = s.stats()
            s.build_list()                        # at the final, dense positions
            start, partners = s.get_list()
            res.append((xs, vs, st, start, partners))
    (x0, v0, s0, st0, p0), (x1, v1, s1, st1, p1) = res
    assert np.diff(st1).max() > kmax0             # the capacity grew during the run
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(v0, v1)
    assert s0 == s1
    np.testing.assert_array_equal(st0, st1)
    ostart, _ = oracle.build_list(oracle.wrap(x1, box), box, rl)
    np.testing.assert_array_equal(st1, ostart)


def test_overflow_in_a_batch_equals_host_loop(ljmd):
    """The same contracting gas in a batch beside a fluid: the graph's rebuild pass
    overflows for the gas only; after the host grows its list, both systems end bit
    for bit where the host-driven loop puts them."""
    n = 1372
    xg, boxg = li.perturbed_fcc(n, 0.0556, 0.1, 706)
    vg = -0.38 * (xg - 0.5 * boxg)
    xf, boxf = li.perturbed_fcc(4000, 0.8442, 0.08, 708)
    vf = li.maxwell_boltzmann(4000, 1.1, 709)
    out = []
    for graph in (0, 1):
        b = ljmd.LJBatch(systems=[(n, boxg, 2.5, 0.3), (4000, boxf, 2.5, 0.3)], precision=ljmd.MD_FP32_FORCE)
        try:
            b.set_tuning(graph=graph)
            b.set_state(0, xg, vg)
            b.set_state(1, xf, vf)
            b.step(300, [0.005, 0.005])
            out.append([b.get_state(k) + (b.stats(k),) for k in range(2)])
        finally:
            b.close()
    for (x0, v0, s0), (x1, v1, s1) in zip(*out):
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(v0, v1)
        assert s0 == s1


def test_nonfinite_stops_graph_loop(ljmd):
    x = li.uniform_positions(500, 20.0, 707)
    v = np.zeros_like(x)
    v[7, 1] = np.inf
    with ljmd.LJSystem(20.0, 500, 2.5, 0.3) as s:
        s.set_tuning(graph=1)
        s.set_state(x, v)
        with pytest.raises(ljmd.MDError) as e:
            s.step(10, 0.005)
        assert e.value.code == ljmd.MD_ERR_NONFINITE

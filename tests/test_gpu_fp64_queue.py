"""The FP64 force loop that classifies listed pairs on the fixed-point shadows and
queues the maybe-inside ones (MD_TUNE_FP64_QUEUE 1, the default) against the plain
loop over the list (0): forces, trajectories and observables equal bit for bit,
for the exact FP64 form and the paper's reciprocal-approximation forms (Sec. 3.3),
in boxes with one cell (every pair a candidate), a dense fluid, the rc = 3.0
cavitation cutoff and a ragged last tile; and both match the oracle."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def cases():
    x, box = li.perturbed_fcc(4001, 0.8442, 0.1, 701)
    yield "fluid-4001", x, box, 2.5
    x, box = li.perturbed_fcc(4 * 9 ** 3, 0.70, 0.1, 702)
    yield "rc3-2916", x, box, 3.0
    x, box = li.perturbed_fcc(300, 0.85, 0.1, 703)       # fewer than 3 cells per axis
    yield "small-box-300", x, box, 2.5
    x, box = li.perturbed_fcc(33, 0.1, 0.2, 704)         # dilute: few pairs inside rc
    yield "dilute-33", x, box, 2.5


CASES = list(cases())


def run(ljmd, x, v, box, rc, precision, queue, steps):
    with ljmd.LJSystem(box, len(x), rc, 0.3, precision) as s:
        s.set_tuning(fp64_queue=queue)
        assert s.get_tuning()["fp64_queue"] == queue
        s.set_state(x, v)
        f0 = s.forces()
        s.step(steps, 0.005)
        xs, vs = s.get_state()
        o = s.observables()
        st = s.stats()
    return f0, xs, vs, o, st


@pytest.mark.parametrize("name,x,box,rc", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["MD_FP64", "MD_FP64_RCP8_CORR", "MD_FP64_RCP23"])
def test_queue_equals_plain_loop_bitwise(ljmd, name, x, box, rc, precision):
    prec = getattr(ljmd, precision)
    v = li.maxwell_boltzmann(len(x), 0.9, 705)
    a = run(ljmd, x, v, box, rc, prec, 1, 80)
    b = run(ljmd, x, v, box, rc, prec, 0, 80)
    np.testing.assert_array_equal(a[0], b[0])   # forces
    np.testing.assert_array_equal(a[1], b[1])   # positions after 80 steps (rebuilds inside)
    np.testing.assert_array_equal(a[2], b[2])   # velocities
    for k in ("pe", "virial", "ke"):
        assert a[3][k] == b[3][k]
    assert a[4]["rebuilds"] == b[4]["rebuilds"] and a[4]["rebuilds"] >= 1


def test_queue_forces_match_oracle(ljmd, oracle):
    """Both loops against the all-pairs oracle (FP64 bar 1e-12, normwise)."""
    for name, x, box, rc in CASES:
        ref = oracle.forces_brute(oracle.wrap(x, box), box, rc)
        rms = np.sqrt((ref ** 2).sum(1).mean())
        for queue in (1, 0):
            with ljmd.LJSystem(box, len(x), rc, 0.3, ljmd.MD_FP64) as s:
                s.set_tuning(fp64_queue=queue)
                s.set_state(x, np.zeros_like(x))
                f = s.forces()
            assert np.abs(f - ref).max() / rms <= 1e-12, (name, queue)


def test_queue_in_a_batch_graph(ljmd):
    """Uneven systems stepped together in graph-captured chunks: the queued loop
    equals the plain loop bit for bit, system by system."""
    systems = li.batch_systems(count=12, seed=706)
    out = []
    for queue in (1, 0):
        b = ljmd.LJBatch(systems=[(c.n, c.box, c.rc, c.skin) for c in systems], precision=ljmd.MD_FP64)
        b.set_tuning(fp64_queue=queue, graph=1)
        for k, c in enumerate(systems):
            b.set_state(k, c.x, c.v)
        b.step(60, [c.dt for c in systems])
        out.append([np.concatenate(b.get_state(k)) for k in range(len(systems))])
        b.close()
    for p, q in zip(*out):
        np.testing.assert_array_equal(p, q)

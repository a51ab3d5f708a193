"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars (written in each test):
  - cell of every particle and pair-list membership: bit-exact at identical
    positions (integer / index results);
  - FP64 forces: max_i |F_i - F_i^ref| / rms_i |F_i^ref| <= 1e-12;
  - FP32-force mode: the same norm <= 1e-5;
  - observables PE, W, KE: relative 1e-12 (FP64 sums in another order);
  - 200-step trajectory: positions within 1e-10 and velocities within 1e-9 of
    the oracle (a 1e-14 perturbation grows to ~1e-13 over these 200 steps in the
    oracle itself), and identical rebuild counts.
"""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def force_err(f, ref):
    rms = np.sqrt((ref ** 2).sum(1).mean())
    return np.abs(f - ref).max() / rms


def sorted_csr(start, partners):
    seg = np.repeat(np.arange(len(start) - 1), np.diff(start))
    order = np.lexsort((partners, seg))
    return partners[order]


def make(ljmd, x, v, box, rc=2.5, skin=0.3, precision=0):
    s = ljmd.LJSystem(box, len(x), rc, skin, precision)
    s.set_state(x, v)
    return s


def configs():
    out = []
    x, box = li.perturbed_fcc(4000, 0.8442, 0.1, 101)
    out.append(("perturbed-4000", x, box))
    x, box = li.perturbed_fcc(4001, 0.8442, 0.1, 102)   # ragged last tile
    out.append(("perturbed-4001", x, box))
    cfg = li.config_small_fluid()
    out.append(("fcc-4000-exact-lattice", cfg.x, cfg.box))   # sites on cell faces
    # a 6^3 lattice exactly on the cell faces (L = 16.8, 6 cells of side 2.8 ->
    # 5 cells of side 3.36), plus points at 0, at the largest double below L and
    # outside the box
    box = 16.8
    g = np.arange(6) * (box / 6)
    pts = np.array([[a, b, c] for a in g for b in g for c in g])
    edge = np.nextafter(box, 0.0)
    extra = np.array([[edge, 1.4, 1.4], [1.4, edge, 4.2], [4.2, 1.4, edge], [-1e-17, 1.4, 9.8],
                      [16.8 + 1.4, 12.6 + 1.4, -1.4], [3.36, 3.36 + 1.4, 1.4]])
    out.append(("cell-faces", np.concatenate([pts, extra]), box))
    x, box = li.perturbed_fcc(518, 0.8442, 0.1, 109)     # exactly 3 cells per axis
    out.append(("three-cells-518", x, box))
    x, box = li.perturbed_fcc(300, 0.85, 0.1, 103)      # fewer than 3 cells per axis
    out.append(("small-box-300", x, box))
    x, box = li.perturbed_fcc(33, 0.1, 0.2, 104)        # one full tile + 1, all pairs
    out.append(("dilute-33", x, box))
    return out


CONFIGS = configs()
IDS = [c[0] for c in CONFIGS]
_U = li.uniform_positions(3000, 18.0, 7)              # uniform, overlaps allowed
LIST_CONFIGS = CONFIGS + [("uniform-3000", _U, 18.0)]
LIST_IDS = IDS + ["uniform-3000"]


def shell_pairs(count=2000, box=300.0, rl=2.8, seed=11):
    """Pairs at distances rl (1 + t), t uniform within three times the widest
    pre-test shell (a few 1e-4 at this L / rl), a fifth of them straddling a
    box face: most pairs fall between the pre-tests' sure-inside and
    sure-outside thresholds, on both sides of rl."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, box, size=(count, 3))
    c[: count // 5, rng.integers(0, 3)] = rng.uniform(0.0, 1.0, size=count // 5)
    u = rng.normal(size=(count, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    t = rng.uniform(-4e-4, 4e-4, size=(count, 1))
    return np.concatenate([c, c + rl * (1.0 + t) * u]), box


# L = 300, and L = 430, the box of the largest system the library takes
# (N = 2^26 - 1 at rho 0.8442), where the float pre-test's shell is widest
# (+-1.6e-4 of rl against +-1.1e-4 at L = 300; the pairs span +-4e-4)
_S = {300: shell_pairs(), 430: shell_pairs(box=430.0, seed=12)}


@pytest.mark.parametrize("box_side", [300, 430])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5],
                         ids=["float", "fixed", "float-pruned", "fixed-pruned", "warp", "staged"])
def test_list_bit_exact_in_the_shell(ljmd, oracle, variant, box_side):
    x, box = _S[box_side]
    with make(ljmd, x, np.zeros_like(x), box) as s:
        s.set_tuning(list_variant=variant)
        s.build_list()
        xw = oracle.wrap(x, box)
        start, partners = s.get_list()
        ostart, opartners = oracle.build_list(xw, box, 2.8)
        assert ostart[-1] > 1000          # many pairs inside, many just outside
        np.testing.assert_array_equal(start, ostart)
        np.testing.assert_array_equal(sorted_csr(start, partners), opartners)


@pytest.mark.parametrize("variant", [0, 4, 5], ids=["lane", "warp", "staged"])
@pytest.mark.parametrize("name,x,box", LIST_CONFIGS, ids=LIST_IDS)
def test_wrap_cells_and_list_bit_exact(ljmd, oracle, name, x, box, variant):
    v = np.zeros_like(x)
    with make(ljmd, x, v, box) as s:
        s.set_tuning(list_variant=variant)
        s.build_list()
        xg, _ = s.get_state()
        xw = oracle.wrap(x, box)
        np.testing.assert_array_equal(xg, xw)      # same wrap, bit for bit
        cell, nc = s.get_cells()
        onc = oracle.cells_per_axis(box, 2.8)
        if onc >= 3:
            assert nc == onc
            np.testing.assert_array_equal(cell, oracle.cell_index(xw, box, 2.8))
        else:
            assert nc == 1 and np.all(cell == 0)
        start, partners = s.get_list()
        ostart, opartners = oracle.build_list(xw, box, 2.8)
        np.testing.assert_array_equal(start, ostart)
        np.testing.assert_array_equal(sorted_csr(start, partners), opartners)


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, FP32_TOL)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,x,box", CONFIGS, ids=IDS)
def test_forces_match_oracle(ljmd, oracle, name, x, box, precision, tol):
    v = np.zeros_like(x)
    with make(ljmd, x, v, box, precision=precision) as s:
        f = s.forces()
    ref = oracle.forces_brute(oracle.wrap(x, box), box, 2.5)
    if np.sqrt((ref ** 2).sum(1).mean()) < 1e-9:   # perfect lattice: forces vanish
        assert np.abs(f).max() < (1e-11 if precision == 0 else 1e-3)
        return
    assert force_err(f, ref) <= tol


def test_forces_rc3_cavitation_cutoff(ljmd, oracle):
    x, box = li.perturbed_fcc(4 * 9 ** 3, 0.70, 0.1, 105)
    for precision, tol in [(0, FP64_TOL), (1, FP32_TOL)]:
        with make(ljmd, x, np.zeros_like(x), box, rc=3.0, precision=precision) as s:
            f = s.forces()
        ref = oracle.forces(x, box, 3.0)
        assert force_err(f, ref) <= tol


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_observables_match_oracle(ljmd, oracle, precision):
    x, box = li.perturbed_fcc(4000, 0.8442, 0.1, 106)
    v = li.maxwell_boltzmann(4000, 0.722, 107)
    with make(ljmd, x, v, box, precision=precision) as s:
        o = s.observables()
    r = oracle.observables(x, v, box, 2.5)
    for k in ["pe", "virial", "ke", "temperature", "pressure"]:
        assert o[k] == pytest.approx(r[k], rel=1e-12), k


def test_full_size_observables(ljmd, oracle):
    """PE, W, KE, T and P of the 2,048,000-particle fluid (FCC 80^3 x 4 displaced by up
    to 0.1, T 0.722) against the oracle's list-based sums, both force forms (the
    observables are FP64 in both): relative 1e-12."""
    x, box = li.perturbed_fcc(2_048_000, 0.8442, 0.1, 112)
    v = li.maxwell_boltzmann(2_048_000, 0.722, 123)
    r = oracle.observables(x, v, box, 2.5)
    for precision in (0, 1):
        with make(ljmd, x, v, box, precision=precision) as s:
            o = s.observables()
        for k in ["pe", "virial", "ke", "temperature", "pressure"]:
            assert o[k] == pytest.approx(r[k], rel=1e-12), (precision, k)


def test_trajectory_200_steps_fp64(ljmd, oracle):
    """The N = 4000 fluid (FCC, rho 0.8442, T 0.722, dt 0.005) for 200 steps."""
    cfg = li.config_small_fluid()
    with make(ljmd, cfg.x, cfg.v, cfg.box) as s:
        s.step(cfg.steps, cfg.dt)
        xg, vg = s.get_state()
        st = s.stats()
        og = s.observables()
    r = oracle.run(cfg.x, cfg.v, cfg.box, cfg.rc, cfg.skin, cfg.steps, cfg.dt)
    d = xg - r["x"]
    d -= cfg.box * np.round(d / cfg.box)
    assert np.abs(d).max() < 1e-10
    assert np.abs(vg - r["v"]).max() < 1e-9
    assert st["rebuilds"] == r["rebuilds"]
    assert st["steps"] == cfg.steps
    ro = oracle.observables(r["x"], r["v"], cfg.box, cfg.rc)
    assert og["pe"] == pytest.approx(ro["pe"], rel=1e-10)


def test_full_size_trajectory_fp64(ljmd, oracle):
    """The 2,048,000-particle fluid (FCC 80^3 x 4, the benchmark's configuration) for 12
    FP64 steps, one list rebuild inside: every position and velocity against the oracle
    (the same bars as the 200-step run), and the same rebuild count."""
    cfg = li.config_large_fluid()
    steps = 12
    with make(ljmd, cfg.x, cfg.v, cfg.box) as s:
        s.step(steps, cfg.dt)
        xg, vg = s.get_state()
        st = s.stats()
    r = oracle.run(cfg.x, cfg.v, cfg.box, cfg.rc, cfg.skin, steps, cfg.dt)
    assert r["rebuilds"] >= 2
    d = xg - r["x"]
    d -= cfg.box * np.round(d / cfg.box)
    assert np.abs(d).max() < 1e-10
    assert np.abs(vg - r["v"]).max() < 1e-9
    assert st["rebuilds"] == r["rebuilds"]


def test_state_into_caller_arrays(ljmd):
    """get_state(out=(x, v)) fills pinned host arrays with the same values as
    get_state()."""
    import torch
    x, box = li.perturbed_fcc(4001, 0.8442, 0.1, 119)
    v = li.maxwell_boltzmann(4001, 0.722, 120)
    with make(ljmd, x, v, box, precision=1) as s:
        s.step(25, 0.005)
        x1, v1 = s.get_state()
        xo = torch.empty((4001, 3), dtype=torch.float64, pin_memory=True).numpy()
        vo = torch.empty((4001, 3), dtype=torch.float64, pin_memory=True).numpy()
        x2, v2 = s.get_state(out=(xo, vo))
        assert x2 is xo and v2 is vo
        np.testing.assert_array_equal(xo, x1)
        np.testing.assert_array_equal(vo, v1)


def test_split_steps_equal_one_call(ljmd):
    """md_step(100) equals md_step(40) + md_step(60) bit for bit (forces kept
    between calls, same rebuild points)."""
    x, box = li.perturbed_fcc(2000, 0.8442, 0.08, 108)
    v = li.maxwell_boltzmann(2000, 0.9, 109)
    for precision in (0, 1):
        with make(ljmd, x, v, box, precision=precision) as a, make(ljmd, x, v, box, precision=precision) as b:
            a.step(100, 0.005)
            b.step(40, 0.005)
            b.step(60, 0.005)
            xa, va = a.get_state()
            xb, vb = b.get_state()
            np.testing.assert_array_equal(xa, xb)
            np.testing.assert_array_equal(va, vb)


def test_fp32_trajectory_close(ljmd, oracle):
    cfg = li.config_small_fluid()
    with make(ljmd, cfg.x, cfg.v, cfg.box, precision=1) as s:
        s.step(20, cfg.dt)
        xg, vg = s.get_state()
    r = oracle.run(cfg.x, cfg.v, cfg.box, cfg.rc, cfg.skin, 20, cfg.dt)
    d = xg - r["x"]
    d -= cfg.box * np.round(d / cfg.box)
    assert np.abs(d).max() < 1e-6
    assert np.abs(vg - r["v"]).max() < 1e-4


def test_list_overflow_grows_capacity(ljmd, oracle):
    """Particles packed into one corner exceed the initial list capacity; the
    library grows it and the list still matches the oracle exactly."""
    box = 20.0
    x = li.uniform_positions(1500, 6.0, 110)
    with make(ljmd, x, np.zeros_like(x), box) as s:
        start, partners = s.get_list()
    ostart, opartners = oracle.build_list(x, box, 2.8)
    np.testing.assert_array_equal(start, ostart)
    np.testing.assert_array_equal(sorted_csr(start, partners), opartners)


def _raw_list(ljmd, x, box, variant, half=False):
    with ljmd.LJSystem(box, len(x), 2.5, 0.3) as s:
        s.set_pair_list(ljmd.MD_LIST_HALF if half else ljmd.MD_LIST_FULL)
        s.set_tuning(list_variant=variant)
        s.set_state(x, np.zeros_like(x))
        s.build_list()
        return s.get_list()


@pytest.mark.parametrize("half", [False, True], ids=["full", "half"])
def test_list_order_equal_across_variants(ljmd, half):
    """Every build variant writes the same partners in the same order (the
    force sums, and so the trajectories, depend on the order), on the wrap and
    cell-face configurations and on corner-packed particles that overflow the
    initial capacity (the list is built again after it grows)."""
    cases = [(n, x, box) for n, x, box in LIST_CONFIGS]
    cases.append(("corner-packed", li.uniform_positions(1500, 6.0, 110), 20.0))
    for name, x, box in cases:
        ref = _raw_list(ljmd, x, box, 0, half)
        for variant in (1, 2, 3, 5) if half else (1, 2, 3, 4, 5):
            got = _raw_list(ljmd, x, box, variant, half)
            np.testing.assert_array_equal(got[0], ref[0], err_msg=f"{name} variant {variant}")
            np.testing.assert_array_equal(got[1], ref[1], err_msg=f"{name} variant {variant}")


def test_single_particle_and_dimer(ljmd, oracle):
    with make(ljmd, np.array([[1.0, 2.0, 3.0]]), np.zeros((1, 3)), 10.0) as s:
        assert np.all(s.forces() == 0.0)
        s.step(3, 0.005)
    x = np.array([[5.0, 5.0, 5.0], [6.1, 5.0, 5.0]])
    with make(ljmd, x, np.zeros_like(x), 10.0) as s:
        f = s.forces()
    np.testing.assert_allclose(f, oracle.forces_brute(x, 10.0, 2.5), rtol=1e-13, atol=1e-15)


def test_errors(ljmd):
    with pytest.raises(ljmd.MDError) as e:
        ljmd.LJSystem(5.0, 100, 2.5, 0.3)          # box < 2 (rc + skin)
    assert e.value.code == ljmd.MD_ERR_ARG
    with pytest.raises(ljmd.MDError) as e:
        ljmd.LJSystem(20.0, 0, 2.5, 0.3)
    assert e.value.code == ljmd.MD_ERR_ARG
    s = ljmd.LJSystem(20.0, 10, 2.5, 0.3)
    with pytest.raises(ljmd.MDError) as e:
        s.step(1, 0.005)                             # no state yet
    assert e.value.code == ljmd.MD_ERR_STATE
    x = li.uniform_positions(10, 20.0, 111)
    v = np.zeros_like(x)
    v[3, 0] = np.nan
    s.set_state(x, v)
    with pytest.raises(ljmd.MDError) as e:
        s.step(2, 0.005)
    assert e.value.code == ljmd.MD_ERR_NONFINITE
    s.close()


def test_full_size_sampled_forces(ljmd, oracle):
    """N = 2,048,000 (FCC 80^3 x 4, rho 0.8442) displaced by up to 0.1: forces of
    400 sampled particles against direct all-pairs sums, both precisions, and
    sum_i F_i ~ 0 over the whole system (full list is symmetric)."""
    x, box = li.perturbed_fcc(2_048_000, 0.8442, 0.1, 112)
    rng = np.random.default_rng(113)
    idx = rng.choice(len(x), size=400, replace=False)
    ref = np.array([oracle.force_on(x, box, 2.5, int(i)) for i in idx])
    rms_ref = np.sqrt((ref ** 2).sum(1).mean())
    for precision, tol in [(0, FP64_TOL), (1, FP32_TOL)]:
        with make(ljmd, x, np.zeros_like(x), box, precision=precision) as s:
            f = s.forces()
            n_list = s.list_size()
        assert np.abs(f[idx] - ref).max() / rms_ref <= tol
        rms = np.sqrt((f ** 2).sum(1).mean())
        assert np.abs(f.sum(0)).max() <= (1e-12 if precision == 0 else 1e-4) * len(x) * rms
        assert 70 * len(x) < n_list < 90 * len(x)


def _pair_keys(start, partners):
    """The pairs of a CSR list as sorted (particle << 32 | partner) keys."""
    seg = np.repeat(np.arange(len(start) - 1, dtype=np.int64), np.diff(start))
    return np.sort((seg << 32) | partners.astype(np.int64))


def test_full_size_list_membership(ljmd, oracle):
    """The benchmark's size, N = 2,048,000 (FCC 80^3 x 4 at rho 0.8442 displaced by up
    to 0.1): every particle's list, built by the default variant, equals the oracle's
    list {j != i : r^2 < rl^2} bit for bit (as sets of caller ids)."""
    x, box = li.perturbed_fcc(2_048_000, 0.8442, 0.1, 116)
    with make(ljmd, x, np.zeros_like(x), box) as s:
        s.build_list()
        start, partners = s.get_list()
    ostart, opartners = oracle.build_list(oracle.wrap(x, box), box, 2.8)
    np.testing.assert_array_equal(start, ostart)
    assert np.array_equal(_pair_keys(start, partners), _pair_keys(ostart, opartners))


def test_cavitation_size_sampled_forces(ljmd, oracle):
    """The cavitation configuration at full size: N = 16,384,000 (FCC 160^3 x 4 at rho
    0.70, displaced by up to 0.1, expanded by 1.05 to rho 0.6047), rc 3.0: forces of
    200 sampled particles against direct all-pairs sums, FP32-force (the form the
    cavitation run uses) and FP64."""
    x, box = li.perturbed_fcc(16_384_000, 0.70, 0.1, 114)
    x *= 1.05
    box *= 1.05
    rng = np.random.default_rng(115)
    idx = rng.choice(len(x), size=200, replace=False)
    xw = oracle.wrap(x, box)
    ref = np.array([oracle.force_on(xw, box, 3.0, int(i)) for i in idx])
    rms_ref = np.sqrt((ref ** 2).sum(1).mean())
    for precision, tol in [(1, FP32_TOL), (0, FP64_TOL)]:
        with make(ljmd, x, np.zeros_like(x), box, rc=3.0, precision=precision) as s:
            f = s.forces()
        assert np.abs(f[idx] - ref).max() / rms_ref <= tol


def test_batched_configuration_forces(ljmd, oracle):
    """The 256-replica configuration (N log-uniform in [500, 32000], rho and T
    uniform) in one arena, after 50 steps (the initial lattices have net forces that
    are small differences of large pair forces, below what FP32 pair arithmetic
    resolves to 1e-5): forces of every eighth system at its current positions
    against the oracle's, both precisions."""
    syss = li.batch_systems(count=256, seed=1004)
    for precision, tol in [(1, FP32_TOL), (0, FP64_TOL)]:
        b = ljmd.LJBatch(systems=[(c.n, c.box, c.rc, c.skin) for c in syss], precision=precision)
        try:
            for k, c in enumerate(syss):
                b.set_state(k, c.x, c.v)
            b.step(50, [c.dt for c in syss])
            for k in range(0, len(syss), 8):
                c = syss[k]
                xk, _ = b.get_state(k)
                f = b.forces(k)
                ref = oracle.forces(xk, c.box, c.rc)
                assert force_err(f, ref) <= tol, k
        finally:
            b.close()


def test_max_size_sampled_forces_and_steps(ljmd, oracle):
    """The largest system the library takes, N = 2^26 - 1 = 67,108,863 (FCC 256^3 x 4 at
    rho 0.8442 less one site, displaced by up to 0.1; the last tile holds 31
    particles): FP32-force forces of 24 sampled particles, the last one among them,
    against direct all-pairs sums; the list size; then 10 steps through the rebuild
    machinery with finite observables. N + 1 is refused."""
    n = ljmd.MD_MAX_N
    x, box = li.perturbed_fcc(n, 0.8442, 0.1, 116)
    rng = np.random.default_rng(117)
    idx = np.concatenate([rng.choice(n - 1, size=23, replace=False), [n - 1]])
    ref = np.array([oracle.force_on(x, box, 2.5, int(i)) for i in idx])
    rms_ref = np.sqrt((ref ** 2).sum(1).mean())
    with make(ljmd, x, np.zeros_like(x), box, precision=1) as s:
        f = s.forces()
        assert np.abs(f[idx] - ref).max() / rms_ref <= FP32_TOL
        assert 70 * n < s.list_size() < 90 * n
        del f
        s.set_state(x, li.maxwell_boltzmann(n, 0.722, 118))
        s.step(10, 0.005)
        o = s.observables()
        assert all(np.isfinite(val) for val in o.values())
        assert s.stats()["steps"] == 10
    with pytest.raises(ljmd.MDError) as e:
        ljmd.LJSystem(box, n + 1, 2.5, 0.3)
    assert e.value.code == ljmd.MD_ERR_ARG

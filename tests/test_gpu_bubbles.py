"""Bubble identification on the GPU (md_bubbles) against the oracle: subcell
counts bit-exact (as the paper's unsigned char), number of bubbles and sizes
equal, on synthetic liquids with carved cavities and on dilute random gases."""
import numpy as np
import pytest

import lj_inputs as li

pytestmark = pytest.mark.gpu


def _carved(cells, rho, radius, centers_frac, seed):
    n = 4 * cells ** 3
    box = li.box_length(n, rho)
    x, _ = li.perturbed_fcc(n, rho, 0.1, seed)
    keep = np.ones(len(x), dtype=bool)
    for cen in np.asarray(centers_frac) * box:
        d = x - cen
        d -= box * np.round(d / box)
        keep &= (d * d).sum(1) > radius ** 2
    return x[keep], box


CASES = [
    ("three-cavities", *_carved(16, 0.70, 4.0, [[0.2, 0.2, 0.2], [0.6, 0.25, 0.7], [0.3, 0.75, 0.55]], 701)),
    ("cavity-across-boundary", *_carved(14, 0.65, 5.0, [[0.0, 0.5, 0.98]], 702)),
    ("dilute-random", li.uniform_positions(3000, 30.0, 703), 30.0),
]


@pytest.mark.parametrize("name,x,box", CASES, ids=[c[0] for c in CASES])
def test_bubbles_match_oracle(ljmd, oracle, name, x, box):
    with ljmd.LJSystem(box, len(x), 3.0, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, np.zeros_like(x))
        g = s.bubbles(3.0, 0.2)
        xw, _ = s.get_state()
    ref = oracle.bubbles(xw, box, 3.0, 0.2)
    assert g["ns"] == ref["ns"]
    np.testing.assert_array_equal(g["counts"], np.minimum(ref["counts"], 255).astype(np.uint8))
    assert g["n_bubbles"] == ref["n_bubbles"]
    np.testing.assert_array_equal(g["sizes"], ref["sizes"])
    if name == "three-cavities":
        assert g["n_bubbles"] == 3


def test_bubbles_in_an_expanded_liquid(ljmd, oracle):
    """The cavitation protocol at 864,000 particles: an FCC 60^3 x 4 lattice at rho
    0.70 with T = 0.9 velocities, expanded by 1.05 per axis (rho 0.605) and run 2000
    FP32-force steps with rc 3.0. Gas subcells then form many clusters of every size;
    counts, cluster count and sizes equal the oracle's at the final positions."""
    n = 864000
    x, box = li.perturbed_fcc(n, 0.70, 0.1, 721)
    v = li.maxwell_boltzmann(n, 0.9, 722)
    x = x * 1.05
    box = box * 1.05
    with ljmd.LJSystem(box, n, 3.0, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, v)
        s.step(2000, 0.005)
        g = s.bubbles(3.0, 0.2)
        xw, _ = s.get_state()
    ref = oracle.bubbles(xw, box, 3.0, 0.2)
    assert ref["n_bubbles"] >= 20
    assert g["ns"] == ref["ns"]
    np.testing.assert_array_equal(g["counts"], np.minimum(ref["counts"], 255).astype(np.uint8))
    assert g["n_bubbles"] == ref["n_bubbles"]
    np.testing.assert_array_equal(g["sizes"], ref["sizes"])


def _mask_particles(gas, ns, side=3.0):
    """Six particles in every liquid subcell of an ns^3 lattice of side `side`
    (count 6 >= 0.2 * 27), none in the gas subcells; pairs no closer than 1.5."""
    off = np.array([[0.5, 0.5, 0.5], [2.0, 0.5, 0.5], [0.5, 2.0, 0.5], [0.5, 0.5, 2.0],
                    [2.0, 2.0, 0.5], [2.0, 0.5, 2.0]])
    liquid = np.flatnonzero(~gas)
    ijk = np.stack([liquid % ns, (liquid // ns) % ns, liquid // (ns * ns)], axis=1).astype(np.float64)
    return (ijk[:, None, :] * side + off[None]).reshape(-1, 3)


@pytest.mark.parametrize("gas_fraction", [0.2, 0.35])
def test_bubbles_on_a_100_cubed_lattice(ljmd, oracle, gas_fraction):
    """The subcell lattice of the cavitation configuration (100^3 subcells of side
    3): a random gas mask at 20 % (many small clusters) and at 35 % (above the
    site-percolation threshold of the simple cubic lattice, 0.31: one cluster spans
    the box, so union-find chains cross every SM). Cluster count and sizes equal
    the oracle's flood fill, and the union-find finishes within its retry bound
    (md_bubbles reports an overrun as an error)."""
    ns = 100
    rng = np.random.default_rng(731 + int(gas_fraction * 100))
    gas = rng.random(ns ** 3) < gas_fraction
    x = _mask_particles(gas, ns)
    box = 3.0 * ns
    with ljmd.LJSystem(box, len(x), 3.0, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, np.zeros_like(x))
        g = s.bubbles(3.0, 0.2)
    k, label = oracle.clusters(gas, ns)
    sizes = np.sort(np.bincount(label[label >= 0])[np.bincount(label[label >= 0]) > 0])[::-1]
    assert g["ns"] == ns
    np.testing.assert_array_equal(g["counts"], np.where(gas, 0, 6).astype(np.uint8))
    assert g["n_bubbles"] == k
    np.testing.assert_array_equal(g["sizes"], sizes)
    if gas_fraction > 0.32:
        assert sizes[0] > 0.5 * gas.sum()   # the spanning cluster

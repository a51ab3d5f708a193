"""Scenarios run by test_gpu_checked.py, once with the product library and once
with the checked build (device bounds checks), each in its own process:

    python tests/checked_scenarios.py {product|checked} OUT.npz

Every hot kernel takes part: binning, the list-build variants, the FP32 and FP64
step kernels (host-driven and graph-captured), the half list, the velocity-bound
rule, observables and pair statistics, an all-pairs box (one cell), a batch with
uneven systems, paused systems and arena reuse, and a checkpoint restore. The
final states go to OUT.npz; any unexpected MDError (MD_ERR_CHECK included) ends
the process with a non-zero status. Last, an out-of-range partner is planted in a
list (checked build only) and must be reported as MD_ERR_CHECK.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lj_inputs as li  # noqa: E402


def main(which: str, out: str) -> None:
    from paper_1210_3450_gb300 import build, ljmd
    path = build.build(checked=(which == "checked"))
    ljmd.load_library(path)
    assert ljmd.version().endswith("checked)") == (which == "checked"), ljmd.version()
    res = {}

    # one system, ragged last tile, both precisions, host-driven and graph-captured
    x, box = li.perturbed_fcc(4001, 0.8442, 0.1, 601)
    v = li.maxwell_boltzmann(4001, 0.9, 602)
    for prec in (ljmd.MD_FP32_FORCE, ljmd.MD_FP64):
        for graph in (0, 1):
            for variant in (0, 3, 4, 5):
                with ljmd.LJSystem(box, 4001, 2.5, 0.3, prec) as s:
                    s.set_tuning(graph=graph, list_variant=variant)
                    s.set_state(x, v)
                    s.step(150, 0.005)
                    o = s.observables()
                    s.pair_stats()
                    xs, vs = s.get_state()
                    res[f"single_p{prec}_g{graph}_v{variant}"] = np.concatenate([xs, vs, s.forces()])
                    res[f"single_p{prec}_g{graph}_v{variant}_obs"] = np.array([o["pe"], o["virial"], o["ke"]])

    # half list and the velocity-bound rule
    for prec in (ljmd.MD_FP32_FORCE, ljmd.MD_FP64):
        with ljmd.LJSystem(box, 4001, 2.5, 0.3, prec) as s:
            s.set_pair_list(ljmd.MD_LIST_HALF)
            s.set_state(x, v)
            s.step(60, 0.005)
            s.observables()
        with ljmd.LJSystem(box, 4001, 2.5, 0.3, prec) as s:
            s.set_validity_rule(ljmd.MD_RULE_DUTC)
            s.set_state(x, v)
            s.step(60, 0.005)
            res[f"dutc_p{prec}"] = np.concatenate(s.get_state())

    # one cell (L = 6.72 < 3 rl): every particle is a candidate
    xa, boxa = li.perturbed_fcc(256, 0.8442, 0.1, 603)
    with ljmd.LJSystem(boxa, 256, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(xa, li.maxwell_boltzmann(256, 0.9, 604))
        s.step(100, 0.005)
        res["one_cell"] = np.concatenate(s.get_state())

    # batch of uneven systems, one paused for a while, one removed and re-added
    specs = [(500, 0.80), (1999, 0.70), (3000, 0.85), (777, 0.60), (6000, 0.75), (1234, 0.80)]
    systems = []
    for k, (n, rho) in enumerate(specs):
        xb, bb = li.perturbed_fcc(n, rho, 0.1, 610 + k)
        systems.append((n, bb, xb, li.maxwell_boltzmann(n, 1.0, 620 + k)))
    b = ljmd.LJBatch(systems=[(n, bb, 2.5, 0.3) for n, bb, _, _ in systems], precision=ljmd.MD_FP32_FORCE)
    try:
        for k, (n, bb, xb, vb) in enumerate(systems):
            b.set_state(k, xb, vb)
        b.step(40, 0.005)
        b.set_active(2, False)
        b.step(30, 0.005)
        b.set_active(2, True)
        b.remove(4)
        n4, bb4, xb4, vb4 = systems[4]
        sid = b.add(n4, bb4, 2.5, 0.3)
        b.set_state(sid, xb4, vb4)
        b.step(50, 0.005)
        for k in range(len(specs)):
            if k == 4:
                continue
            res[f"batch_{k}"] = np.concatenate(b.get_state(k))
        res["batch_new"] = np.concatenate(b.get_state(sid))
    finally:
        b.close()

    # checkpoint and restore
    with ljmd.LJSystem(box, 4001, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, v)
        s.step(37, 0.005)
        ck = s.checkpoint()
        s.step(20, 0.005)
        a1 = np.concatenate(s.get_state())
        s.restore(ck)
        s.step(20, 0.005)
        a2 = np.concatenate(s.get_state())
        assert np.array_equal(a1, a2)
        res["checkpoint"] = a2

    # an out-of-range partner planted in a list: the checked build's pair loop
    # skips it and reports MD_ERR_CHECK, now and at every later call; the product
    # build refuses to write list words
    with ljmd.LJSystem(box, 4001, 2.5, 0.3, ljmd.MD_FP32_FORCE) as s:
        s.set_state(x, v)
        s.step(1, 0.005)
        if which == "checked":
            s.debug_set_list_word(5, 0, 4001 + 7)
            for _ in range(2):
                try:
                    s.step(1, 0.005)
                    raise AssertionError("planted list word not reported")
                except ljmd.MDError as e:
                    assert e.code == ljmd.MD_ERR_CHECK, e
                    assert "check bits 32" in str(e), e
        else:
            try:
                s.debug_set_list_word(5, 0, 4001 + 7)
                raise AssertionError("the product build wrote a list word")
            except ljmd.MDError as e:
                assert e.code == ljmd.MD_ERR_ARG, e

    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])

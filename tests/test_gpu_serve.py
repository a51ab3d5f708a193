"""Serving: runs that arrive while others are on the GPU are admitted as arena
space frees up, advance together, and each result is bit-for-bit the result of
the same run alone (FP32-force mode, the serving default)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", ["shared", "srpt"])
def test_served_results_equal_alone(ljmd, policy):
    from paper_1210_3450_gb300 import serve
    reqs = []
    rng = np.random.default_rng(5)
    for k in range(10):
        n = int(rng.integers(300, 5000))
        reqs.append(serve.Request(id=k, arrival=0.002 * k, n=n, rho=float(rng.uniform(0.6, 0.85)),
                                  temperature=float(rng.uniform(0.72, 1.2)),
                                  steps=int(rng.integers(30, 150)), seed=1000 + k))
    # budget for roughly three of these runs at a time: later ones must wait
    budget = 3 * 5000 * 900
    srv = serve.MDServer(budget, precision=ljmd.MD_FP32_FORCE, chunk=40, keep_state=True, policy=policy,
                         active_particles=6000)
    try:
        summary = srv.run(reqs)
    finally:
        srv.close()
    assert summary["completed"] == len(reqs)
    waited = [r for r in srv.done if r.admitted > min(q.finished for q in srv.done)]
    assert waited, "the budget should have made some requests wait for space"
    assert all(r.finished >= r.admitted >= r.arrival for r in srv.done)
    for r in srv.done:
        x0, v0 = serve.initial_state(r)
        with ljmd.LJSystem(r.box, r.n, r.rc, r.skin, ljmd.MD_FP32_FORCE) as s:
            s.set_state(x0, v0)
            s.step(r.steps, r.dt)
            x, v = s.get_state()
            o = s.observables()
            st = s.stats()
        np.testing.assert_array_equal(r.result["x"], x)
        np.testing.assert_array_equal(r.result["v"], v)
        assert r.result["pe"] == o["pe"] and r.result["ke"] == o["ke"]
        assert r.result["rebuilds"] == st["rebuilds"]


def test_request_larger_than_arena_is_rejected(ljmd):
    from paper_1210_3450_gb300 import serve
    r = serve.Request(id=0, arrival=0.0, n=200000, rho=0.8, temperature=1.0, steps=10, seed=1)
    srv = serve.MDServer(10_000_000, precision=ljmd.MD_FP32_FORCE)
    try:
        s = srv.run([r])
    finally:
        srv.close()
    assert s["rejected"] == 1 and s["completed"] == 0


def test_cancelled_requests_free_their_space(ljmd):
    """Clients cancel two runs (one soon after arrival, one later): neither
    completes, their arena space returns, and every other run completes with the
    result it has alone."""
    from paper_1210_3450_gb300 import serve
    reqs = [serve.Request(id=k, arrival=0.001 * k, n=1500 + 300 * k, rho=0.8, temperature=1.0,
                          steps=400, seed=2000 + k) for k in range(6)]
    reqs[1].cancel_after = 0.0
    reqs[3].steps = 1_000_000          # still running when it is cancelled
    reqs[3].cancel_after = 0.2
    srv = serve.MDServer(3 * 3500 * 900, precision=ljmd.MD_FP32_FORCE, chunk=20)
    try:
        summary = srv.run(reqs)
        assert srv.batch.usage()["systems_used"] == 0
    finally:
        srv.close()
    assert summary["cancelled"] == 2 and summary["completed"] == 4
    for r in srv.done:
        if r.id in (1, 3):
            assert r.result == {"cancelled": True}
            continue
        x0, v0 = serve.initial_state(r)
        with ljmd.LJSystem(r.box, r.n, r.rc, r.skin, ljmd.MD_FP32_FORCE) as s:
            s.set_state(x0, v0)
            s.step(r.steps, r.dt)
            o = s.observables()
        assert r.result["pe"] == o["pe"] and r.result["ke"] == o["ke"]


def test_zero_budget_is_refused(ljmd):
    from paper_1210_3450_gb300 import serve
    with pytest.raises(ljmd.MDError) as e:
        serve.MDServer(0, precision=ljmd.MD_FP32_FORCE)
    assert e.value.code == ljmd.MD_ERR_ARG


def test_served_large_and_growing_runs_equal_alone(ljmd, oracle):
    """Requests of the served workload's sizes: one with N = 120,000 and, arriving
    while others run, a droplet (an FCC block at density 0.85 in a box at 0.3)
    whose pair lists need more room than its density-based capacity, so the
    server's arena grows its list while the other runs share the arena. Every
    result equals the same run alone bit for bit."""
    from paper_1210_3450_gb300 import serve
    drop = serve.Request(id=3, arrival=0.02, n=20_000, rho=0.3, temperature=0.9, steps=90, seed=3003,
                         layout="droplet")
    # precondition: the droplet's longest list exceeds the capacity its footprint gives
    x0, _ = serve.initial_state(drop)
    start, _ = oracle.build_list(x0, drop.box, drop.rc + drop.skin)
    f = ljmd.footprint(drop.n, drop.box, drop.rc, drop.skin)
    kmax0 = f["list_words"] // (((drop.n + 31) // 32) * 32)
    assert np.diff(start).max() > kmax0
    reqs = [serve.Request(id=0, arrival=0.0, n=120_000, rho=0.8, temperature=0.9, steps=3000, seed=3000),
            serve.Request(id=1, arrival=0.0, n=3000, rho=0.7, temperature=1.1, steps=150, seed=3001),
            serve.Request(id=2, arrival=0.01, n=8000, rho=0.65, temperature=0.8, steps=120, seed=3002),
            drop]
    rng = np.random.default_rng(3010)
    for k in range(4, 10):
        reqs.append(serve.Request(id=k, arrival=0.06 + 0.01 * k, n=int(rng.integers(1000, 20000)),
                                  rho=float(rng.uniform(0.6, 0.85)), temperature=float(rng.uniform(0.72, 1.2)),
                                  steps=int(rng.integers(40, 120)), seed=3000 + k))
    srv = serve.MDServer(200_000_000, precision=ljmd.MD_FP32_FORCE, chunk=20, keep_state=True)
    try:
        summary = srv.run(reqs)
    finally:
        srv.close()
    assert summary["completed"] == len(reqs)
    # the droplet joined while the big run was on the device
    big = next(r for r in srv.done if r.id == 0)
    d = next(r for r in srv.done if r.id == 3)
    assert d.admitted < big.finished
    for r in srv.done:
        x0, v0 = serve.initial_state(r)
        with ljmd.LJSystem(r.box, r.n, r.rc, r.skin, ljmd.MD_FP32_FORCE) as s:
            s.set_state(x0, v0)
            s.step(r.steps, r.dt)
            x, v = s.get_state()
            o = s.observables()
            st = s.stats()
        np.testing.assert_array_equal(r.result["x"], x)
        np.testing.assert_array_equal(r.result["v"], v)
        assert r.result["pe"] == o["pe"] and r.result["ke"] == o["ke"]
        assert r.result["rebuilds"] == st["rebuilds"]

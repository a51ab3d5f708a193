"""Multi-GPU runs are independent replicas (no data exchange on the path): the
whole-job value is the work of all ranks over the slowest rank's time. The
cross-rank reduction of bench.py is exercised here with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        sec, units = bench.replica_totals(dist, 1.0 + rank, 100.0 * (rank + 1))
        q.put((rank, sec, units))
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, sec, units in got:
        assert sec == 2.0            # the slowest rank's time
        assert units == 300.0        # every rank's work


def test_replica_totals_single_process():
    import bench
    assert bench.replica_totals(None, 1.5, 10.0) == (1.5, 10.0)

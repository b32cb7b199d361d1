"""Replica aggregation across ranks (gloo, two CPU processes)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_1002_3028_gb300 import replicas

    replicas.init("gloo")
    assert replicas.world() == (world, rank, rank)
    replicas.barrier()
    ms, units = replicas.combine(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    out.put((rank, ms, units))
    replicas.finish()


def test_two_ranks_take_the_slowest_time_and_the_summed_units():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_single_rank_is_the_identity():
    from paper_1002_3028_gb300 import replicas

    assert replicas.combine(12.5, 7.0) == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0

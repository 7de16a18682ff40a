"""The benchmark's multi-rank path on CPU: two gloo ranks (one process per GPU
in production), barrier, max over ranks of the timed region, whole-job rate of
independent replicas; the reference arm prints on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    value, ms_max = bench.aggregate_rate(1_000_000, ms_local, world)
    q.put((rank, value, ms_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max in out:
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 1_000_000 / 0.150)


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup = 1, 0

    bench.reference_arm(A())
    assert capsys.readouterr().out == ""

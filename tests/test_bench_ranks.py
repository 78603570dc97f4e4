"""The N > 1 path of bench.py (independent replicas, one per rank) with two gloo ranks on
the CPU: every rank gets the slowest rank's time, and the whole-job value counts the solves
of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 100.0 * (rank + 1)  # rank 1 is the slow one
    value, t_ms = bench.replica_value(t_local, 5, world, "cpu")
    slowest = bench.max_over_ranks(float(rank), world, "cpu")
    out.put((rank, value, t_ms, slowest))
    dist.destroy_process_group()


def test_replica_value_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for rank, value, t_ms, slowest in got:
        assert t_ms == 200.0 and slowest == 1.0
        assert value == pytest.approx(2 * 5 / 0.2)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.replica_value(250.0, 5, 1, "cpu") == (20.0, 250.0)

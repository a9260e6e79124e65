"""Multi-GPU runs are independent replicas (the grid is not sharded): the
benchmark's barrier, max-over-ranks timing and whole-job value, exercised
with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = 100.0 + 50.0 * rank          # the slower replica sets the time
    m = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.replica_value(world, 1000, 10, m)
    q.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    import torch.multiprocessing as mp
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
    assert [o[1] for o in out] == [150.0, 150.0]
    # 2 replicas x 1000 nodes x 10 steps in 150 ms
    assert abs(out[0][2] - 2 * 1000 * 10 / 0.150 / 1e6) < 1e-12

"""The multi-rank path of the benchmark on CPU: two gloo ranks, each with its
own batch (replicas, no collective on the data path); the reported time is
the slowest rank's and the value counts the units of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    t_max = bench.max_over_ranks(t_local, "cpu")
    value = bench.weak_scaling_value(1000, 4, t_max, world)
    q.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    # 2 ranks x 1000 units x 4 steps over 0.15 s
    assert res[0][2] == pytest.approx(2 * 1000 * 4 / 0.15)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.weak_scaling_value(10, 2, 1000.0, 1) == pytest.approx(20.0)

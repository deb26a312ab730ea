"""The multi-rank path of the benchmark on CPU: two gloo ranks, each timing an independent replica,
agree on the job's time (the slowest rank's) and on the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    m = bench.max_over_ranks(ms, world)
    out[rank] = (m, bench.replica_rate(1 << 20, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()  # no fork of a possibly threaded process
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    m, rate = out[0]
    assert m == 15.0
    assert rate == pytest.approx((1 << 20) * 2 / 15e-3 / 1e9)


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_rate(1 << 28, 1, 1.0) == pytest.approx(268.435456)

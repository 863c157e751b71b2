"""The multi-GPU path of bench.py is replicas only: each rank solves its own problems, the job
time is the maximum over ranks and the value counts every rank's solves. The aggregation is
checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]               # rank 1 is the slow one
    value, ms_max = bench.replica_throughput(local_ms, steps=5, world=world, dist=dist,
                                             device="cpu")
    dist.barrier()
    out[rank] = (value, ms_max)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, ms_max = res[rank]
        assert ms_max == 250.0
        assert value == pytest.approx(2 * 5 / 0.25)


def test_single_rank_needs_no_collective():
    import bench
    value, ms_max = bench.replica_throughput(200.0, steps=4, world=1, dist=None, device="cpu")
    assert ms_max == 200.0 and value == pytest.approx(20.0)

"""The N > 1 path of bench.py runs one independent replica of the workload per rank: timings are
reduced with a max over ranks and the job's time per load step counts every rank's steps.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = bench.max_over_ranks([1.0 + rank, 10.0 - rank])
        out[rank] = mx + [bench.replica_value(mx[0], 17, world)]
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_value_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        assert res[rank][:2] == [2.0, 10.0]
        assert res[rank][2] == pytest.approx(2.0 / (17 * 2))


def test_single_process_is_identity():
    assert bench.max_over_ranks([3.5, 1.25]) == [3.5, 1.25]
    assert bench.replica_value(3.4, 17, 1) == pytest.approx(0.2)

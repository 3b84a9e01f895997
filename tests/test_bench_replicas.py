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


def test_oracle_sample_on_several_cores_tiny_workload():
    """The all-core oracle timing runs the same sample (one full Newton iteration of load step 1) in one
    single-thread process per core and averages their times (2 processes on a 2-subdomain case here);
    a load step is Newton iterations x that iteration plus the commit."""
    s = bench.oracle_sample_all_cores("tiny2_1x1x2", n_proc=2)
    assert s is not None and s["cores"] == 2
    for k in bench.SAMPLE_KEYS:
        assert s[k] > 0.0
    assert s["newton_s"] >= s["assembly_s"] + s["setup_s"]
    v = bench.oracle_step_seconds(s, 2.5)
    assert v == pytest.approx(2.5 * s["newton_s"] + s["commit_s"])


def test_algorithmic_fapply_counts_band_entries():
    """One 8^3 box: 2187 dofs, half bandwidth 275 -> 2187 x 276 entries, 4 flops and 16 bytes each."""
    import workloads as W
    w = W.cube("one_box", 8, 1)
    a = bench.algorithmic_fapply(w)
    assert a["factor_entries"] == 2187 * 276
    assert a["flops"] == 4.0 * 2187 * 276 and a["bytes"] == 16.0 * 2187 * 276
    assert bench.algorithmic_fapply(W.CUBE64)["factor_entries"] == 512 * 2187 * 276

"""The N>1 host logic of bench.py (replicas: one realization stream per
rank, timing = max over ranks, value = all ranks' voxels / that time),
exercised by two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        p = bench.rank_workload(rank, 400)
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        mx = bench.max_over_ranks(ms, world, torch.device("cpu"))
        value = bench.job_rate(p["nx"] * p["ny"] * p["nz"] * 5, world, mx)
        seeds = [None] * world
        dist.all_gather_object(seeds, p["seed"])
        out[rank] = (mx, value, tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for mx, value, seeds in res.values():
        assert mx == 150.0                                   # the slowest rank
        assert value == pytest.approx(400**3 * 5 * 2 / 0.150)  # all ranks' voxels
        assert len(set(seeds)) == world                      # independent realizations


def test_single_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.job_rate(1000, 1, 1000.0) == 1000.0

"""Host logic of the multi-GPU benchmark path, run as two gloo ranks on the CPU:
each rank takes its own independent volume, timings reduce to the slowest rank,
and the job's throughput counts every rank's units over that time."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench._dist()
        local_ms = 100.0 + 37.5 * rank  # rank 1 is the slower one
        t_max = bench._max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ws, r, t_max, bench._job_value(ws, 1e9, t_max * 1e-3), bench._workload_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (ws, r, t_max, value, seed) in res.items():
        assert ws == world and r == rank
        assert t_max == 137.5  # both ranks see the slower rank's time
        assert value == pytest.approx(2 * 1e9 / 0.1375 / 1e9)
    assert res[0][4] != res[1][4]  # independent volumes per rank


def test_single_process_needs_no_collective():
    assert bench._max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench._job_value(1, 8e9, 2.0) == 4.0

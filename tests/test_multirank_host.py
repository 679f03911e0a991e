"""The N-GPU host logic of bench.py, run as two gloo ranks on the CPU: the step
time is the maximum over the ranks and the throughput counts every rank's pixels
(replicas of the workload, weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.job_ms(ms_by_rank[rank], world, torch.device("cpu"))
    out[rank] = (ms, bench.job_value(816_000, ms, world))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_time_is_the_max_over_ranks_and_value_counts_all_ranks(world):
    port = _free_port()
    ms_by_rank = [0.70, 0.85][:world]
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, ms_by_rank, out), nprocs=world, join=True)
    for r in range(world):
        ms, v = out[r]
        assert ms == pytest.approx(max(ms_by_rank))
        assert v == pytest.approx(world * 816_000 / (max(ms_by_rank) * 1e-3) / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_ms(0.5, 1) == 0.5
    assert bench.job_value(816_000, 0.5, 1) == pytest.approx(1632.0)

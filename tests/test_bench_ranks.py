"""The replica form of bench.py on two gloo ranks (CPU): whole-job figures take the slowest rank's
times and the sum of the ranks' work, and only rank 0 runs the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        # rank r: its own step time, TR time and work
        res = bench.combine_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), 2.0 + rank, 7 * (rank + 1), world,
                                  device="cpu")
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_max_time_and_sum_work():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):  # every rank sees the same whole-job figures
        assert out[r] == (15.0, 3000.0, 3.0, 21.0)


def test_one_rank_passes_through():
    assert bench.combine_ranks(12.5, 40, 1.5, 9, 1) == (12.5, 40.0, 1.5, 9.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        workload = "tiny-50kbp-10x"
        steps = 1
        warmup = 0
    assert bench.reference_arm(Args(), 1, 2) is None
    assert capsys.readouterr().out == ""

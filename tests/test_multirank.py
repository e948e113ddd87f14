"""The multi-rank path of the benchmark on CPU (gloo, two ranks).

With N GPUs every rank sweeps its own replica (the strips of one problem are not
split across GPUs), so the only cross-rank steps are the barrier around the timed
region and the maximum of the ranks' times; the reference arm runs on rank 0 only.
"""
import os
import socket
import types

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(torch, dist, world, 100.0 + 25.0 * rank, device="cpu")
        out[rank] = (ms, bench.job_rate(world, 1_000_000, 4, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_whole_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, rate = res[rank]
        assert ms == 125.0  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1_000_000 * 4 / 0.125)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = types.SimpleNamespace(ref_nt=1, steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""

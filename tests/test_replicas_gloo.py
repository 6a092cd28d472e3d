"""Host logic of the multi-GPU bench path (replicas: every rank runs the
whole workload, the job's step time is the slowest rank's, throughput adds up),
exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, l = bench.dist_env()
        ms = bench.replica_time(1.0 + rank, w)  # rank 1 is the slow one
        out[rank] = (r, w, l, ms, bench.job_rate(1000, ms, w))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_add_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, l, ms, rate) in res.items():
        assert (r, w, l) == (rank, world, rank)
        assert ms == 2.0  # max over ranks
        assert rate == pytest.approx(1000 * 2 / 2e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.replica_time(1.5, 1) == 1.5
    assert bench.job_rate(10 ** 9, 1.0, 1) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        gpus, steps, warmup = 2, 1, 0

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""

"""The multi-GPU path of bench.py is replicas (one process per GPU, no data
exchange); its host logic -- the slowest rank's time, the whole-job rate and
rank 0 alone printing the reference arm -- checked with world-size-2 gloo
process groups on the CPU."""
import json
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        out[rank] = (ms, bench.whole_job_rate(1000, world, 4, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms, rate = out[rank]
        assert ms == 15.0                       # the slowest rank
        assert rate == 1000 * 2 * 4 / 0.015     # both ranks' rows, slowest time


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 1, 2, 1000.0) == 20.0


def test_reference_arm_only_rank0_prints(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(args, bench.full_sizes(True)) == 0
    assert capsys.readouterr().out == ""

"""The multi-GPU path is replicas (one independent amplitude stream per
rank, no data-path collective): the host logic that splits the work and
combines the timing runs here as two gloo ranks on CPU."""
import os
import socket

import numpy as np
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]          # the second rank is slower
        total, value = bench._whole_job(local_ms, 40, world)
        bits = bench._bitstrings(1000 + rank, 5)  # each rank's own bitstrings
        out.put((rank, total, value, [b.tolist() for b in bits]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, b0), (r1, t1, v1, b1) = res
    assert t0 == t1 == 150.0                      # max over ranks
    assert v0 == v1 == pytest.approx(2 * 40 / 0.150)   # whole-job amplitudes/s
    assert b0 != b1                               # different work per rank


def test_single_process_needs_no_process_group():
    total, value = bench._whole_job(200.0, 10, 1)
    assert total == 200.0 and value == pytest.approx(50.0)

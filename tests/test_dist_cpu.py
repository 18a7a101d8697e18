"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2): each
rank steps its own replica (distinct seeds, no collective on the data path),
the job time is the slowest rank's, and the whole-job value counts the work
of every rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = [120.0, 150.0][rank]
    job_ms = bench.max_over_ranks(ms, dist)
    units = 1000 * (rank + 1)
    total = torch.tensor([units], dtype=torch.float64)
    dist.all_reduce(total)
    out[rank] = (job_ms, bench.scene_seed("cloth_stack", rank), float(total.item()) / (job_ms / 1e3))
    dist.destroy_process_group()


def test_two_rank_gloo_bookkeeping():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] != out[1][1]
    assert abs(out[0][2] - 3000 / 0.15) < 1e-6


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.scene_seed("cloth_stack", 0) == 2 and bench.scene_seed("wires", 1) == 2

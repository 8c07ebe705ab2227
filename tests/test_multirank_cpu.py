"""The multi-rank path on the host: two gloo ranks, each its own independent
agent (Philox key (seed, rank), buffer drawn with seed offset rank), the
barrier and the max-over-ranks timing reduction that bench.py uses.  No GPU:
the agents' work is the oracle's relabel draw."""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
from paper_2408_11052_gb300 import workload


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workload.SMALL_FP32.with_(E=4, T=40, B=16)
        obs, act, done = workload.buffer_contents(w, n=40, mean_len=8.0, seed_offset=rank)
        buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
        buf.insert(obs, act, done)
        _, _, _, idx = oracle.relabel.sample_relabel(buf, w.seed, rank, 3, w.B, w.goals(), w.gamma)
        bench.barrier(world)
        local = 10.0 + rank                       # a per-rank "elapsed time"
        mx = bench.max_over_ranks(local, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, np.asarray(idx).tolist())
        out[rank] = (mx, gathered)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_independent_agents_and_max_reduction():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(rank_main, args=(world, free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        mx, gathered = out[r]
        assert mx == 11.0                          # max over ranks, seen by every rank
        assert gathered == out[0][1]               # the same all-gathered draws on every rank
    idx0, idx1 = np.array(out[0][1][0]), np.array(out[0][1][1])
    assert idx0.shape == idx1.shape == (16, 3)
    assert not np.array_equal(idx0, idx1)          # independent agents draw independent batches

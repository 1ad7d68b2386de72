"""The multi-GPU path of bench.py on CPU: two gloo ranks, disjoint noise vectors, the slowest
rank's time, whole-job throughput (no GPU: the ranks exchange only their timing)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle import core as oc


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank], dist)
    dist.barrier()
    out[rank] = t
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    times = [123.0, 456.0]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    assert out[0] == out[1] == 456.0
    assert bench.aggregate_rate(world, 48, 3, 456.0) == pytest.approx(2 * 48 * 3 / 0.456)


def test_ranks_draw_disjoint_noise_vectors():
    nhit, steps = 16, 5
    offs = {r: [bench.rank_hit_offset(r, nhit, k) for k in range(steps)] for r in range(4)}
    hits = [o + j for r in offs for o in offs[r] for j in range(nhit)]
    assert len(hits) == len(set(hits))  # no Philox counter is used twice
    a = oc.noise_packed(2, bench.rank_hit_offset(0, nhit, 0), 1, 1200)
    b = oc.noise_packed(2, bench.rank_hit_offset(1, nhit, 0), 1, 1200)
    assert abs(np.vdot(a, b)) < 5 * np.sqrt(1200)  # independent vectors

"""The multi-GPU path of bench.py is replicas only: every rank decodes its own
seeded frames and ranks exchange nothing but the timing (max over ranks).
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
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
        seeds = [bench.replica_seed(rank, b, f, 4, 16) for b in range(4) for f in range(16)]
        slowest = bench.max_over_ranks(1.0 + rank)
        out[rank] = (seeds, slowest)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_decode_disjoint_frames_and_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    s0, t0 = res[0]
    s1, t1 = res[1]
    assert len(set(s0)) == len(s0) == 64
    assert not set(s0) & set(s1)
    assert t0 == t1 == 2.0


def test_single_process_max_is_identity():
    assert bench.max_over_ranks(3.5) == 3.5

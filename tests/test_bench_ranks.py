"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own timing,
agree on the slowest rank's time (the replicas exchange nothing else)."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu", world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, "cpu", 1) == 3.25

"""Multi-process logic of bench.py on CPU (gloo, world size 2): the job time is the slowest rank's
time on every rank, and every GPU of a node tunes into its own cache file."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 30.25][rank]
        out[rank] = bench._max_over_ranks(local_ms, dist, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_max_over_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 30.25, 1: 30.25}


def test_single_process_keeps_its_time_and_ranks_get_their_own_tune_cache():
    assert bench._max_over_ranks(7.0, None, "cpu") == 7.0
    paths = {bench._tune_cache_path(r) for r in range(8)}
    assert len(paths) == 8

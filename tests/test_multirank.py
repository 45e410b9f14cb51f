"""Replica path of bench.py on CPU: two gloo ranks, each with its own
configuration, combine timings by max and share no data-path collective."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cfg = bench.config_for_rank(rank, "flux4")
    fingerprint = float(np.abs(cfg["U"]).sum() + cfg["U"][0, 0, 0, 0].real)
    ms = bench.max_over_ranks(10.0 + rank)
    fp = [None] * world
    dist.all_gather_object(fp, fingerprint)
    out[rank] = (ms, fp, cfg["dims"])
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 11.0  # max over ranks
    fp = out[0][1]
    assert fp[0] != fp[1]  # each rank has its own configuration
    assert tuple(out[0][2]) == tuple(out[1][2]) == (4, 4, 4, 4)

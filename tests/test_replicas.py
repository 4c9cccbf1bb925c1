"""Multi-GPU replica logic on CPU: two gloo ranks (no GPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2408_11988_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, lr = replicas.world()
    t = 1.0 + r                      # rank r "took" 1 + r seconds
    tmax = replicas.max_over_ranks(t, dist)
    seed = replicas.replica_seed(100, r)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    out[rank] = (ws, r, lr, tmax, replicas.job_rate(10, ws, tmax), tuple(seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ws, r, lr, tmax, rate, seeds = out[rank]
        assert (ws, r, lr) == (world, rank, rank)
        assert tmax == 2.0                      # the slowest rank's time
        assert rate == pytest.approx(10 * 2 / 2.0)
        assert len(set(seeds)) == world and seeds[0] == 100


def test_single_process_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.world() == (1, 0, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(6, 1, 2.0) == 3.0

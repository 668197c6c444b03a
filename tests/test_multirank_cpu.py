"""The multi-rank host logic of bench.py on CPU with two gloo ranks: every rank draws its own
independent layers (weak scaling), the step time is the max over ranks, and the whole-job
rate counts the units of all ranks over the slowest rank's time. No data-path collective."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import lfa_workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lay = W.layers("conv64_k3_n32")[0]
    w = W.weights(lay, seed=bench.rank_seed(lay, rank))
    ms = [1.0 + rank, 10.0 - rank]                       # per-rank timings
    red = bench.reduce_max(ms, dist)
    digest = torch.tensor([float(np.sum(w.astype(np.float64)))])
    gathered = [torch.zeros(1) for _ in range(world)]
    dist.all_gather(gathered, digest)
    out[rank] = (red, [float(g) for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        red, sums = out[rank]
        assert red == [2.0, 10.0]                        # max over ranks
        assert sums[0] != sums[1]                        # distinct per-rank layers
    lay = W.layers("conv64_k3_n32")[0]
    rate = bench.aggregate_rate(lay.n_sigma, 10, world, 20.0)
    assert rate == pytest.approx(world * lay.n_sigma * 10 / 0.020)


def test_single_rank_reduce_is_identity():
    assert bench.reduce_max([3.0, 1.5]) == [3.0, 1.5]

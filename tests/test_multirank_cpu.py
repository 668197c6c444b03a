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


# ----------------------------------------------------------------------------- frequency shards
def _shard_worker(rank, world, port, out):
    """One rank of a frequency-sharded job: its share of the half grid comes from the library's
    partition (lfa_options_t.shard_rank / shard_count); its dL/dw is the oracle's backward over the
    share and its conjugates; one all-reduce sums the ranks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2506_05617_gb300 import lfa as C
    n, m = 6, 5
    w = W.weights(W.Layer(3, 4, 3, 3, n, m, "normal", 2.0, 77))
    F_h, first, count = C.lfa_debug_shard_range(n, m, rank, world)
    half = O.half_grid(n, m)
    share = half[first:first + count]
    fc = ((-(share // m)) % n) * m + ((-(share % m)) % m)
    freqs = np.unique(np.concatenate([share, fc]))            # the share and its conjugates
    s, U, V = O.lfa_svd(w, n, m, compute_uv=True)
    g = W.upstream_gradient((n * m, 3), seed=5).astype(np.float64)
    part = O.lfa_backward(w, n, m, g[freqs], U[freqs], V[freqs], freqs=freqs)
    t = torch.from_numpy(part.copy())
    dist.all_reduce(t)                                        # the job's one data-path collective
    ranges = [None] * world
    dist.all_gather_object(ranges, (first, count))
    out[rank] = (F_h, ranges, t.numpy(), O.lfa_backward(w, n, m, g, U, V))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_frequency_shards_cover_the_half_grid_once_and_sum_to_the_backward(world):
    from paper_2506_05617_gb300 import build as B
    B.build()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        F_h, ranges, dw_sum, dw_full = out[rank]
        cover = np.zeros(F_h, int)
        for first, count in ranges:
            cover[first:first + count] += 1
        assert np.all(cover == 1)                               # every half-grid frequency exactly once
        assert all(ranges[i][0] + ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))  # rank order
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1                  # balanced
        np.testing.assert_allclose(dw_sum, dw_full, rtol=1e-12, atol=1e-12)


def test_shard_range_rejects_invalid_arguments():
    from paper_2506_05617_gb300 import lfa as C
    assert C.lfa_debug_shard_range(4, 4, 2, 2)[0] == -1
    assert C.lfa_debug_shard_range(4, 4, 0, 0)[0] == -1
    assert C.lfa_debug_shard_range(4, 4, 0, 1) == (10, 0, 10)

"""Multi-rank paths emulated with gloo ranks on the CPU (world size 2).

1. Sharded edges (the one exchange step of a multi-GPU split of a single graph): every rank
   resamples and splats its own edges; an integer sum all-reduce of the partial histogram
   stacks must give the single-device histogram bit for bit (integer addition is exact and
   order-free), and, since the box passes are linear, smoothing the reduced histogram equals
   reducing the ranks' smoothed partial sums.
2. Independent graphs per rank (what bench.py runs for N > 1): the job time is the slowest
   rank's, the updates are summed.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graph():
    rng = np.random.default_rng(77)
    E, G = 301, 3
    src = rng.uniform(5, 90, (E, 2))
    dst = rng.uniform(5, 70, (E, 2))
    group = rng.integers(0, G, E).astype(np.int32)
    weight = rng.integers(1, 4, E).astype(np.int32)
    return src, dst, group, weight, G, 80, 96


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle

    src, dst, group, weight, G, H, W = _graph()
    mine = np.arange(len(src)) % world == rank          # this rank's edges
    off, xy = oracle.straight_polylines(src[mine], dst[mine])
    r_off, r_xy = oracle.resample(off, xy, 0, 24, 2.0)
    part = oracle.splat(r_off, r_xy, group[mine], weight[mine], G, H, W)
    hist = torch.from_numpy(part.copy())
    dist.all_reduce(hist, op=dist.ReduceOp.SUM)          # the exchange step
    sums_part = torch.from_numpy(oracle.smooth(part, 3, 3))
    dist.all_reduce(sums_part, op=dist.ReduceOp.SUM)

    import bench

    ms, upd = bench.reduce_over_ranks(dist, 10.0 + rank, 100.0 * (rank + 1), device="cpu")
    if rank == 0:
        np.save(out + "_hist.npy", hist.numpy())
        np.save(out + "_sums.npy", sums_part.numpy())
        np.save(out + "_red.npy", np.array([ms, upd]))
    dist.destroy_process_group()


def test_sharded_histogram_allreduce_is_exact(tmp_path, oracle_mod):
    out = str(tmp_path / "r")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    src, dst, group, weight, G, H, W = _graph()
    off, xy = oracle_mod.straight_polylines(src, dst)
    r_off, r_xy = oracle_mod.resample(off, xy, 0, 24, 2.0)
    full = oracle_mod.splat(r_off, r_xy, group, weight, G, H, W)
    np.testing.assert_array_equal(np.load(out + "_hist.npy"), full)
    np.testing.assert_array_equal(np.load(out + "_sums.npy"), oracle_mod.smooth(full, 3, 3))
    ms, upd = np.load(out + "_red.npy")
    assert ms == 11.0 and upd == 300.0

"""Multi-rank logic on CPU ranks (gloo, world size 2), no GPU.

1. The sharded form of one resample: every rank holds a slice of the
   weights; an all-reduce gives max and sum (hence B, Eq. 3), an all-gather
   gives every rank the whole vector (any particle may propose any index),
   each rank runs the chains of its own particles, and the slices joined
   together equal the unsharded oracle bit for bit.
2. The benchmark's replica aggregation: the slowest rank's time and the
   particles of all ranks.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synthetic

WORLD = 2
N = 3000 + 7
Y = 2.5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sharded_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w_all = synthetic.gaussian_weights(N, Y, 17)
        lo, hi = rank * N // world, (rank + 1) * N // world
        w_local = torch.from_numpy(w_all[lo:hi].copy())
        # all-reduce of (max, sum) -> B on every rank
        mx = w_local.max().clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = torch.tensor([float(w_local.double().sum())], dtype=torch.float64)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        r = (float(sm.item()) / N) / float(mx.item())
        B = int(math.ceil(math.log(0.01) / math.log1p(-r)))
        # all-gather of the weights (slices of unequal length)
        sizes = [(k + 1) * N // world - k * N // world for k in range(world)]
        padded = torch.zeros(max(sizes), dtype=torch.float32)
        padded[: w_local.numel()] = w_local
        parts = [torch.zeros(max(sizes), dtype=torch.float32) for _ in range(world)]
        dist.all_gather(parts, padded)
        w_full = np.concatenate([parts[k][: sizes[k]].numpy() for k in range(world)])
        for variant in (oracle.MEGOPOLIS, oracle.METROPOLIS):
            anc = oracle.resample(w_full, B, 9, variant, i0=lo, i1=hi)
            np.save(os.path.join(out_dir, "anc_%d_%d.npy" % (variant, rank)), anc)
        np.save(os.path.join(out_dir, "B_%d.npy" % rank), np.array([B]))
    finally:
        dist.destroy_process_group()


def _replica_worker(rank, world, port, out_dir):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank
        ms, particles = bench.replica_aggregate(local_ms, 1000 * (rank + 1), dist, "cpu")
        np.save(os.path.join(out_dir, "rep_%d.npy" % rank), np.array([ms, particles]))
    finally:
        dist.destroy_process_group()


def test_sharded_resample_equals_unsharded(tmp_path):
    mp.start_processes(_sharded_worker, args=(WORLD, _free_port(), str(tmp_path)),
                       nprocs=WORLD, start_method="spawn")
    w_all = synthetic.gaussian_weights(N, Y, 17)
    st, B_ref, q = oracle.compute_B(w_all, 0.01)
    Bs = [int(np.load(tmp_path / ("B_%d.npy" % k))[0]) for k in range(WORLD)]
    assert Bs[0] == Bs[1]
    assert Bs[0] == B_ref or abs(q - round(q)) < 1e-9 * q
    for variant in (oracle.MEGOPOLIS, oracle.METROPOLIS):
        joined = np.concatenate([np.load(tmp_path / ("anc_%d_%d.npy" % (variant, k)))
                                 for k in range(WORLD)])
        assert np.array_equal(joined, oracle.resample(w_all, Bs[0], 9, variant))


def test_replica_aggregation_takes_slowest_rank(tmp_path):
    mp.start_processes(_replica_worker, args=(WORLD, _free_port(), str(tmp_path)),
                       nprocs=WORLD, start_method="spawn")
    for k in range(WORLD):
        ms, particles = np.load(tmp_path / ("rep_%d.npy" % k))
        assert ms == 15.0 and particles == 3000

"""The multi-rank benchmark logic on CPU: two gloo ranks (no GPU).

Each rank runs its own batch (weak scaling, no data-path collective); the
step time is the maximum over ranks and the whole-job value counts every
rank's units.  The oracle stands in for the per-rank computation so that
ranks' results can be checked independently."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_1401_6238_gb300 import workloads as wl
    b = wl.batched_square(count=6, seed=bench.rank_seed(rank), n_lo=8, n_hi=24)
    ys = []
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        ys.append(oracle.fast_y(h, [x] * (m - 1), [n] * m).real)
    step = 0.010 * (rank + 1)  # rank 1 is the slow one
    slowest = bench.max_over_ranks(step, dist, "cpu")
    rate = bench.aggregate_rate(world, len(b), slowest)
    out[rank] = (b.dims.tolist(), float(np.concatenate(ys).sum()), slowest, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
    (d0, s0, t0, r0), (d1, s1, t1, r1) = out[0], out[1]
    assert d0 != d1 and s0 != s1          # each rank has its own batch
    assert t0 == t1 == pytest.approx(0.020)  # max over ranks
    assert r0 == r1 == pytest.approx(2 * 6 / 0.020)

"""Multi-GPU form of the bench: independent replicas (weak scaling), no
data-path collective.  The host-side logic -- rank-dependent right-hand
sides, barrier, max-over-ranks timing and the whole-job aggregate -- runs
here as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    wl = dict(bench.WORKLOADS["c2"], n=16)
    f = bench.make_rhs(wl, 2, bench.rank_seed(wl, rank))
    bench.barrier(w)
    my_ms = 100.0 * (rank + 1)            # pretend per-rank timed region
    mx = bench.reduce_max(my_ms, w)
    out[rank] = (mx, float(f.sum()))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 200.0          # max over ranks
    assert out[0][1] != out[1][1]                   # each rank solves its own batch
    assert bench.aggregate(256, world, 5, 200.0) == pytest.approx(256 * 2 * 5 / 0.2)


def test_single_process_defaults():
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)

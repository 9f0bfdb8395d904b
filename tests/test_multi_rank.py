"""The multi-rank (torchrun) host logic of bench.py on CPU with the gloo backend, world size 2:
each rank gets its own seeded units (replica inputs, or its own batch of problems) and the job's
step time is the slowest rank's.  No GPU and no data-path collective are involved."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import workloads
    r, w, _ = bench._env_rank()
    bench._dist_init(w, backend="gloo")
    bench._barrier(w)
    slowest = bench._max_over_ranks(10.0 + 3.0 * r, w)
    sizes = workloads.batched_sizes(16, seed=bench._rank_seed(3, r))
    pts, _ = workloads.stokes_uniform(64, seed=bench._rank_seed(1, r))
    out[r] = (slowest, sizes, pts.sum())
    dist.destroy_process_group()


def test_two_ranks_partition_the_units_and_report_the_slowest():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 13.0          # max over ranks of 10 and 13
    assert res[0][1] != res[1][1]                  # each rank has its own batch of problems
    assert res[0][2] != res[1][2]                  # and its own replica inputs
    assert all(1024 <= n <= 65536 for r in res for n in res[r][1])

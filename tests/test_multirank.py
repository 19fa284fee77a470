"""The multi-GPU path shards independent scenes across ranks with no data
exchange; only the timing maximum and the point total are reduced.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, n = bench.aggregate(10.0 + 5.0 * rank, 1000 + rank, dist, "cpu")
    frames, offsets, eps, cfg = bench.make_workload("batched", rank, 2, n_scenes=3)
    out[rank] = (ms, n, float(frames[0].sum()), int(offsets[-1]))
    dist.destroy_process_group()


def test_two_rank_aggregation_and_independent_shards():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (ms0, n0, s0, t0), (ms1, n1, s1, t1) = out[0], out[1]
    assert ms0 == ms1 == 15.0                      # slowest rank
    assert n0 == n1 == 2001                        # all ranks' points
    assert s0 != s1                                # each rank runs its own seeded scenes


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.aggregate(3.5, 42) == (3.5, 42)

"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): ranks
build independent key sets (weak scaling, no data-path collective) and the
job time is the maximum over ranks."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import shk_inputs

    dist.init_process_group("gloo", rank=rank, world_size=ws, init_method=f"tcp://127.0.0.1:{port}")
    t = bench.max_over_ranks(float(rank + 1) * 0.5, dist, "cpu")
    seed = bench.rank_key_seed(rank)
    keys = shk_inputs.distinct_u64(2000, seed)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, seed, keys.tolist()))


def test_two_gloo_ranks_take_max_time_and_disjoint_keys():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [1.0, 1.0]
    assert out[0][2] != out[1][2]
    a, b = set(out[0][3]), set(out[1][3])
    assert len(a) == len(b) == 2000 and not (a & b)

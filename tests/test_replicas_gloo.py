"""Multi-GPU runs are replicas only: each rank solves its own seeded instance and the bench
reports the slowest rank's time. The host side of that (per-rank seeds, max over ranks, one
printing rank) runs here on CPU with two gloo ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    L = bench.replica_layout("c1", rank)
    r, c, v = synth.generate(L)
    t = 10.0 + 5.0 * rank  # this rank's timed region
    tmax = bench.reduce_max(t, dist, "cpu")
    out.put((rank, int(L.seed), int(len(r)), float(np.sum(v)), tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_seed_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, n0, v0, m0), (r1, s1, n1, v1, m1) = res
    assert (r0, r1) == (0, 1)
    assert s1 == s0 + 1  # distinct seeded instances
    assert v0 != v1
    assert m0 == m1 == 15.0  # both ranks see the slowest rank's time


def test_reduce_max_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5

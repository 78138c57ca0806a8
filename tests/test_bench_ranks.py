"""The multi-rank path of bench.py on CPU: two gloo ranks run the same
helpers the benchmark runs under torchrun (one process per GPU).  A single
chain does not shard, so the ranks are replicas: each advances its own chain
from its own seed, and they meet only at the barriers around the timed
region and at the max-over-ranks of the times.  The reference arm runs on
rank 0 alone; the other ranks return without work."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.sync_ranks(dist)
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")          # rank 1 is the slower one
        seed = bench.replica_seed(rank)
        m0 = synth.initial_mps_entries(seed, 12, 4)
        bench.sync_ranks(dist)
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            if rank != 0:
                bench.run_reference(bench.parse([]))
        q.put((rank, t, seed, float(np.sum(m0 ** 2)), out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, n0, o0), (r1, t1, s1, n1, o1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.5                      # every rank reports the slowest
    assert s0 != s1 and n0 != n1                # independent replicas
    assert o1 == ""                             # reference arm: rank 1 does no work


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    bench.sync_ranks(None)
    assert bench.replica_seed(0) != bench.replica_seed(1)

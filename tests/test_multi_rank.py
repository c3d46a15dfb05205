"""The N>1 path of bench.py on CPU: two gloo ranks, each with its own
independent batch of replicas (seed + rank, no data-path collective); the
timing reduction takes the maximum over ranks and the hop count the sum."""
import os

import pytest


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    from paper_2004_09081_gb300 import workloads
    ws, r, local = bench.dist_setup(False)
    wl = workloads.batched_batio3(0 + r)
    sig = tuple((rep.cells[0], rep.n_vac, rep.n_H, round(rep.T, 6)) for rep in wl.replicas[:4])
    t = bench.allreduce_max(1.5 + r, ws, "cpu")
    h = bench.allreduce_sum(100.0 * (r + 1), ws, "cpu")
    bench.barrier(ws)
    q.put((r, sig, t, h))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_replicas_and_reduce_timing():
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, sig0, t0, h0), (r1, sig1, t1, h1) = out
    assert sig0 != sig1           # each rank draws its own replicas
    assert t0 == t1 == 2.5        # max over ranks
    assert h0 == h1 == 300.0      # hops summed over ranks

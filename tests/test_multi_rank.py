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


def test_parallel_oracle_timing_matches_serial_runs():
    """The host-parallel CPU baseline: worker processes run the oracle as it
    stands on their share of the replicas; with a budget that admits one run
    per replica, the summed hop count equals the serial runs' exactly."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    from oracle import timing
    from paper_2004_09081_gb300 import workloads
    wl = workloads.batched_batio3(0)
    wl.replicas = [r for r in wl.replicas if r.cells[0] <= 20][:3]
    jobs = bench.oracle_jobs(wl, 0)
    rate, hops, secs, done, procs = timing.parallel_rate(jobs, 2, 1e-9, cores=3)
    assert procs == 3 and done == 3 and rate > 0
    want = 0
    for j in jobs:
        L = oracle.Lattice(j["cells"], j["nf"], j["n_vac"], j["n_H"], seed=0, replica=j["r"])
        L.set_rates(j["Ea_O"], j["Ea_H"], j["T"], Ez=j["Ez"], a_ang=j["a"], cap_v=j["cap"],
                    n_tau=j["n_tau"], precision=j["precision"])
        L.run(2)
        want += L.counters()["hops"]
    assert hops == want

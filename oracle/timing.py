"""The oracle timed on independent replicas in parallel worker processes
(TEST INFRASTRUCTURE: only the benchmark's CPU-baseline and reference legs use
this module).

The oracle runs as it stands: one serial lattice per process, nothing tuned.
The replicas of a batch are independent lattices, so N worker processes on N
host cores give the oracle's throughput on the whole host.  Workers are fresh
interpreters (exec'd, not forked), which is safe after the parent process has
initialised CUDA.
"""
from __future__ import annotations

import os
import time


def replica_job(r, cells, nf, n_vac, n_H, T, Ea_O, Ea_H, Ez, a, cap, precision, seed, n_Fe=0, site=None,
                n_tau=1.0):
    """One replica's parameters as a plain dict (what a worker needs to build it)."""
    return {"r": int(r), "cells": tuple(int(c) for c in cells), "nf": tuple(int(f) for f in nf),
            "n_vac": int(n_vac), "n_H": int(n_H), "T": float(T), "Ea_O": float(Ea_O), "Ea_H": float(Ea_H),
            "Ez": float(Ez), "a": float(a), "cap": int(cap), "precision": int(precision), "seed": int(seed),
            "n_Fe": int(n_Fe), "site": site, "n_tau": float(n_tau)}


def run_jobs(jobs, windows, budget_s):
    """Run the listed replicas `windows` windows each, cycling through the list
    until `budget_s` seconds of run time are spent.  Only kmc runs are timed
    (not building the lattices).  Returns (hops, seconds, replica runs)."""
    import oracle
    hops, secs, done, i = 0, 0.0, 0, 0
    while jobs and secs < budget_s:
        j = jobs[i % len(jobs)]
        i += 1
        L = oracle.Lattice(j["cells"], j["nf"], j["n_vac"], j["n_H"], seed=j["seed"], replica=j["r"],
                           n_Fe=j["n_Fe"])
        if j["site"]:
            L.set_site_energy(vv=j["site"]["vv"], fe=j["site"]["fe"])
        L.set_rates(j["Ea_O"], j["Ea_H"], j["T"], Ez=j["Ez"], a_ang=j["a"], cap_v=j["cap"],
                    n_tau=j.get("n_tau", 1.0), precision=j["precision"])
        t0 = time.perf_counter()
        L.run(windows)
        secs += time.perf_counter() - t0
        hops += L.counters()["hops"]
        done += 1
    return hops, secs, done


def _worker():
    """Entry point of a worker process: jobs as JSON on stdin, result on stdout."""
    import json
    import sys
    req = json.loads(sys.stdin.read())
    print(json.dumps(run_jobs(req["jobs"], req["windows"], req["budget_s"])))


def parallel_rate(jobs, windows, budget_s, cores=None):
    """Throughput of the oracle over `jobs` on `cores` processes (default: every
    host core): the replicas are dealt round-robin to the workers, each runs
    its share for `budget_s` seconds; hops/s = all hops / the longest worker's
    run time.  Returns (hops/s, hops, seconds, replica runs, processes)."""
    import json
    import subprocess
    import sys

    import oracle
    oracle.build()  # once, before the workers load the library
    cores = max(1, min(cores or os.cpu_count() or 1, len(jobs)))
    parts = [jobs[k::cores] for k in range(cores)]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = f"import sys; sys.path.insert(0, {root!r}); from oracle.timing import _worker; _worker()"
    procs = [subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True)
             for _ in parts]
    for pr, part in zip(procs, parts):
        pr.stdin.write(json.dumps({"jobs": part, "windows": windows, "budget_s": budget_s}))
        pr.stdin.close()
    res = []
    for pr in procs:
        out = pr.stdout.read()
        if pr.wait() != 0:
            raise RuntimeError("oracle worker failed")
        res.append(json.loads(out))
    hops = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    done = sum(r[2] for r in res)
    return (hops / secs if secs > 0 else 0.0), hops, secs, done, cores

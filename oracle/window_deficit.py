"""Writes the windowing-error table the autotuner's accuracy bound reads.

TEST INFRASTRUCTURE / CALIBRATION: runs only the oracle, on the CPU.

The synchronous-sublattice windows are an approximation of the serial kMC of
Sec. II.A (a vacancy that crosses into a fragment whose colour already ran
loses the rest of its window; one fragment is exact).  This script measures
that error as the hop-rate deficit 1 - H_window / H_BKL: the same lattice and
initial state run for the same simulated time by the windowed oracle and by
the oracle's conventional BKL (Sec. II.A).  Rows: actual fragment edge e
(lattice L = 4e cells, 4^3 fragments, so every edge is exactly e), n_tau of
the window tau = n_tau / (8 k_fast), and two compositions spanning the
batched hydride workload (BaTiO3, barriers 0.70 / 0.35 eV): vacancies only,
and x = 0.3 H- per cell, where H- exchanges set k_fast.

    python -m oracle.window_deficit            # writes the table (a few minutes, all cores)
"""
from __future__ import annotations

import json
import math
import multiprocessing as mp
import os
import sys

EDGES = (4, 5, 6, 7, 8)
N_TAU = (0.25, 0.5, 1.0, 2.0)
COMPOSITIONS = {"vacancies_only": {"x": 0.0, "T": 800.0, "seeds": 4},
                "hydride_x0.3": {"x": 0.3, "T": 650.0, "seeds": 16}}
N_VAC = 96
HOPS_PER_SEED = 250_000
OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2004_09081_gb300",
                   "window_deficit.json")


def _lattice(e, comp, seed):
    import oracle
    L = 4 * e
    nh = int(math.floor(comp["x"] * L**3 + 0.5))
    lat = oracle.Lattice((L, L, L), (4, 4, 4), N_VAC, nh, seed=seed)
    return lat


def _job(args):
    e, cname, n_tau, seed = args
    comp = COMPOSITIONS[cname]
    # window length of the run: enough windows for HOPS_PER_SEED hops
    probe = _lattice(e, comp, seed)
    probe.set_rates(0.70, 0.35, comp["T"], a_ang=4.01, n_tau=n_tau, precision=0)
    probe.run(40)
    per_window = max(probe.counters()["hops"] / 40.0, 1e-3)
    W = int(min(max(HOPS_PER_SEED / per_window, 200), 400_000))
    win = _lattice(e, comp, seed)
    win.set_rates(0.70, 0.35, comp["T"], a_ang=4.01, n_tau=n_tau, precision=0)
    win.run(W)
    t = W * win.params()["tau"]
    ref = _lattice(e, comp, seed)
    ref.set_rates(0.70, 0.35, comp["T"], a_ang=4.01, n_tau=n_tau, precision=0)
    ref.bkl_run(t, stream=seed)
    return (e, cname, n_tau, seed, win.counters()["hops"], ref.counters()["hops"])


def main():
    jobs = [(e, c, nt, s) for e in EDGES for c in COMPOSITIONS for nt in N_TAU
            for s in range(COMPOSITIONS[c]["seeds"])]
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count()) as pool:
        res = pool.map(_job, jobs, chunksize=1)
    table = {}
    for e in EDGES:
        for c in COMPOSITIONS:
            for nt in N_TAU:
                rows = [r for r in res if r[:3] == (e, c, nt)]
                hw = sum(r[4] for r in rows)
                hb = sum(r[5] for r in rows)
                per = [1.0 - r[4] / r[5] for r in rows]
                mean = sum(per) / len(per)
                # standard error from the scatter over seeds: hops of one lattice
                # are correlated (a vacancy next to an H- swaps back and forth),
                # so counting statistics would understate it
                se = math.sqrt(sum((d - mean) ** 2 for d in per) / (len(per) - 1) / len(per))
                table.setdefault(str(e), {}).setdefault(c, {})[str(nt)] = {
                    "deficit": 1.0 - hw / hb, "se": se, "per_seed": per, "hops_window": hw, "hops_bkl": hb}
    doc = {
        "what": "hop-rate deficit 1 - H_window/H_BKL of the windowed fragment scheme against the serial BKL "
                "of Sec. II.A, same lattice, same initial state, same simulated time",
        "rows": "fragment edge (cells) -> composition -> n_tau",
        "lattice": "L = 4 e cells (4^3 fragments of edge e), 96 vacancies, BaTiO3 a = 4.01 A, "
                   "barriers 0.70 / 0.35 eV, plain FP64 oracle",
        "compositions": COMPOSITIONS,
        "error": "se = standard error of the per-seed deficits",
        "command": "python -m oracle.window_deficit",
        "table": table,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)
    for e in EDGES:
        print(e, {c: {nt: "%.4f+-%.4f" % (table[str(e)][c][str(nt)]["deficit"], table[str(e)][c][str(nt)]["se"])
                      for nt in N_TAU} for c in COMPOSITIONS})


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()

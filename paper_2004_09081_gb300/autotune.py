"""Launch-configuration autotuner, subject to an accuracy bound.

Knobs:

  edge         target fragment edge in cells, 4..8 (the partition gives each
               dimension an even fragment count nearest L/edge)
  n_tau        window length tau = n_tau / (8 k_fast), n_tau in {0.25, 0.5, 1, 2}
  schedule     0: replica-resident kernel where the state fits one SM,
               1: colour-phase kernels for every replica
  cluster_top  how many of the largest replicas run as 2-CTA clusters
               (-1: SMs/8, 0: none)

Warps per CTA follow from the replica's shared-memory class in the resident
kernel (128, 256 or 1024 threads) and are not searched.

Accuracy: the synchronous-sublattice windows approximate the serial kMC of
Sec. II.A; a vacancy that crosses into a fragment whose colour already ran
loses the rest of its window.  ``window_deficit.json`` (written by the
oracle, ``python -m oracle.window_deficit``) tables that error as the hop-rate
deficit against the serial BKL, by fragment edge and n_tau.  A candidate is
accepted when the deficit at the smallest fragment edge of any replica of the
batch is at most ``bound`` (1%) for every tabled composition whose estimate
is resolved (deficit above twice its standard error); unresolved rows must be
consistent with the bound within two standard errors.  Among the accepted
candidates the one with the highest hops per second of device time wins.
"""
from __future__ import annotations

import json
import os

from . import fkmc

_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "window_deficit.json")

EDGES = (4, 5, 6, 7, 8)
N_TAUS = (0.25, 0.5, 1.0, 2.0)
LAUNCH = ({"schedule": 0, "cluster_top": -1}, {"schedule": 0, "cluster_top": 0})


def deficit_table(path: str = _TABLE) -> dict:
    with open(path) as f:
        return json.load(f)["table"]


def smallest_edge(cells, edge: int) -> int:
    """The shortest fragment edge over the dimensions of one lattice."""
    return min(L // fkmc.kmc_partition_count(L, edge) for L in cells)


def window_deficit(table: dict, edge: int, n_tau: float):
    """Deficit estimates {composition: (deficit, se)} at a fragment edge: the
    tabled edge itself, else interpolated linearly in 1/edge between the two
    nearest tabled edges (below the smallest tabled edge: scaled as 1/edge from
    it; above the largest: its value, which bounds the smaller deficit)."""
    tabled = sorted(int(e) for e in table)
    key = str(float(n_tau))
    out = {}
    for comp in table[str(tabled[0])]:
        def at(e):
            row = table[str(e)][comp][key]
            return row["deficit"], row["se"]
        if edge in tabled:
            out[comp] = at(edge)
        elif edge < tabled[0]:
            d, s = at(tabled[0])
            out[comp] = (d * tabled[0] / edge, s * tabled[0] / edge)
        elif edge > tabled[-1]:
            out[comp] = at(tabled[-1])
        else:
            lo = max(e for e in tabled if e < edge)
            hi = min(e for e in tabled if e > edge)
            f = (1.0 / lo - 1.0 / edge) / (1.0 / lo - 1.0 / hi)
            (dl, sl), (dh, sh) = at(lo), at(hi)
            out[comp] = (dl + f * (dh - dl), sl + f * (sh - sl))
    return out


def accepted(est: dict, bound: float) -> bool:
    for d, se in est.values():
        if d > 2.0 * se:          # resolved: the estimate itself must meet the bound
            if d > bound:
                return False
        elif d - 2.0 * se > bound:  # unresolved: not inconsistent with the bound
            return False
    return True


def batch_deficit(table, cells, edge, n_tau):
    """Deficit estimates at the shortest fragment edge of any replica of the
    batch (the largest error): (largest point estimate, that edge, estimates
    by composition)."""
    e_min = min(smallest_edge(c, edge) for c in cells)
    est = window_deficit(table, e_min, n_tau)
    return max(v[0] for v in est.values()), e_min, est


def autotune(cells, comps, seed, Ea_O, Ea_H, T, *, field_z=0.0, precision=fkmc.FKMC_MIXED, bound=0.01,
             edges=EDGES, n_taus=N_TAUS, launch=LAUNCH, warm_windows=2, timed_windows=8, **batch_kw):
    """Return (best candidate, results).  Each result is a dict with the
    candidate, its deficit estimate, whether it met the bound and (if it did)
    hops per second of device time over a short timed run through the ABI."""
    table = deficit_table()
    geom = [(c[0], c[1], c[2]) for c in cells]
    results = []
    for edge in edges:
        for n_tau in n_taus:
            worst, e_min, est = batch_deficit(table, geom, edge, n_tau)
            ok = accepted(est, bound)
            for lo in launch:
                cand = {"edge": edge, "n_tau": n_tau, **lo}
                res = {"candidate": cand, "at_edge": e_min, "accepted": ok, "hops_per_s": None,
                       "deficit": {k: {"deficit": v[0], "se": v[1]} for k, v in est.items()}}
                if ok:
                    kw = dict(batch_kw)
                    kw.update(cand)
                    b = fkmc.Batch(cells, comps, seed, precision=precision, **kw)
                    try:
                        b.set_barriers(Ea_O, Ea_H, T, field_z=field_z)
                        b.run(warm_windows)
                        # the same simulated time at every n_tau
                        s = b.run(max(1, int(round(timed_windows / n_tau))))
                        res["hops_per_s"] = s.hops / (s.gpu_ms / 1e3) if s.gpu_ms > 0 else 0.0
                        res["cap_v"] = b.info(0).cap_v
                    finally:
                        b.close()
                results.append(res)
    timed = [r for r in results if r["hops_per_s"]]
    if not timed:
        raise RuntimeError("no candidate meets the accuracy bound")
    best = max(timed, key=lambda r: r["hops_per_s"])["candidate"]
    return best, results

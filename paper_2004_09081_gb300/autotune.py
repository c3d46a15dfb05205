"""Launch-configuration autotuner: fragment edge, schedule and cluster pairing.

Each candidate builds the batch with its options, runs a few warm-up windows
and then a short timed run through the C ABI; the candidate with the highest
hops per second of device time wins.  The knobs:

  edge         fragment edge in cells (changes the fragmentation, so candidates
               are different, equally valid realisations of the windowed
               method; smaller edges cross more fragment boundaries per hop,
               whose O(tau) windowing error is characterised in the tests)
  schedule     0: replica-resident kernel where the state fits one SM,
               1: colour-phase kernels for every replica
  cluster_top  how many of the largest replicas run as 2-CTA clusters
               (-1: SMs/8, 0: none)

Warps per CTA follow from the replica's shared-memory class (128, 256 or 1024
threads) and are not searched.
"""
from __future__ import annotations

from . import fkmc

DEFAULT_CANDIDATES = (
    {"edge": 4, "schedule": 0, "cluster_top": -1},
    {"edge": 4, "schedule": 0, "cluster_top": 0},
    {"edge": 5, "schedule": 0, "cluster_top": -1},
    {"edge": 6, "schedule": 0, "cluster_top": -1},
    {"edge": 4, "schedule": 1, "cluster_top": 0},
)


def autotune(cells, comps, seed, Ea_O, Ea_H, T, *, field_z=0.0, precision=fkmc.FKMC_MIXED,
             candidates=DEFAULT_CANDIDATES, warm_windows=2, timed_windows=8, **batch_kw):
    """Return (best candidate dict, list of (candidate, hops/s, cap_v))."""
    results = []
    for cand in candidates:
        kw = dict(batch_kw)
        kw.update(cand)
        b = fkmc.Batch(cells, comps, seed, precision=precision, **kw)
        try:
            b.set_barriers(Ea_O, Ea_H, T, field_z=field_z)
            b.run(warm_windows)
            s = b.run(timed_windows)
            rate = s.hops / (s.gpu_ms / 1e3) if s.gpu_ms > 0 else 0.0
            results.append((dict(cand), rate, b.info(0).cap_v))
        finally:
            b.close()
    best = max(results, key=lambda x: x[1])[0]
    return best, results

"""Launch-configuration autotuner (the fragment edge and the schedule).

Each candidate builds the batch with its options, runs a few warm-up windows
and then a short timed run through the C ABI; the candidate with the highest
hops per second of device time wins.  The candidates change the
fragmentation, so they are different (equally valid) realisations of the
windowed method: the choice is a speed/accuracy knob, recorded with the
result.  Smaller edges cross more fragment boundaries per hop, whose O(tau)
windowing error is characterised in the test-suite; the default candidates
stay within 4..6 cells.
"""
from __future__ import annotations

from . import fkmc

DEFAULT_CANDIDATES = ({"edge": 4, "schedule": 0}, {"edge": 5, "schedule": 0}, {"edge": 6, "schedule": 0})


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

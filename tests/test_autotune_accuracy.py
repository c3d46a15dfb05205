"""The autotuner's accuracy bound (no GPU): the windowing-deficit table the
oracle wrote, its use by fragment edge and n_tau, and its reproduction by the
oracle.

The synchronous-sublattice windows approximate the serial kMC of Sec. II.A: a
vacancy that crosses into a fragment whose colour already ran loses the rest
of its window.  The table holds that error as the hop-rate deficit against the
oracle's serial BKL; the autotuner accepts a (fragment edge, n_tau) only where
it is at most 1%.
"""
import math

import pytest


@pytest.fixture(scope="module")
def at():
    from paper_2004_09081_gb300 import _build, autotune, fkmc
    _build.build()
    fkmc.load()
    return autotune


def test_table_has_every_candidate(at):
    t = at.deficit_table()
    for e in at.EDGES:
        for comp in ("vacancies_only", "hydride_x0.3"):
            for nt in at.N_TAUS:
                row = t[str(e)][comp][str(float(nt))]
                assert math.isfinite(row["deficit"]) and row["se"] > 0
                assert row["hops_window"] > 0 and row["hops_bkl"] > 0


def test_vacancy_deficit_grows_with_the_window_and_shrinks_with_the_edge(at):
    """The error vanishes as tau -> 0 and falls as fragments grow (fewer
    boundary crossings per hop): monotone within two standard errors."""
    t = at.deficit_table()
    for e in at.EDGES:
        rows = [t[str(e)]["vacancies_only"][str(float(nt))] for nt in at.N_TAUS]
        for a, b in zip(rows, rows[1:]):
            assert b["deficit"] > a["deficit"] - 2 * math.hypot(a["se"], b["se"])
        assert rows[-1]["deficit"] > rows[0]["deficit"]
    for nt in (1.0, 2.0):
        d4 = t["4"]["vacancies_only"][str(nt)]
        d8 = t["8"]["vacancies_only"][str(nt)]
        assert d8["deficit"] < d4["deficit"]


def test_interpolation_and_bound(at):
    t = at.deficit_table()
    exact = at.window_deficit(t, 6, 1.0)
    assert exact["vacancies_only"][0] == t["6"]["vacancies_only"]["1.0"]["deficit"]
    # between tabled edges: between their values
    lo = t["5"]["vacancies_only"]["2.0"]["deficit"]
    hi = t["6"]["vacancies_only"]["2.0"]["deficit"]
    assert at.window_deficit(t, 5, 2.0)["vacancies_only"][0] == lo
    # below the table (edge 2, 3 of uneven partitions): larger than at edge 4
    assert at.window_deficit(t, 3, 1.0)["vacancies_only"][0] > t["4"]["vacancies_only"]["1.0"]["deficit"]
    assert min(lo, hi) <= at.window_deficit(t, 6, 2.0)["vacancies_only"][0] <= max(lo, hi)
    # the bound
    assert at.accepted({"a": (0.005, 0.001)}, 0.01)
    assert not at.accepted({"a": (0.02, 0.001)}, 0.01)
    assert at.accepted({"a": (0.012, 0.01)}, 0.01)       # unresolved, consistent with the bound
    assert not at.accepted({"a": (0.05, 0.02)}, 0.01)    # resolved, above


def test_the_batched_workload_at_the_former_default_fails_the_bound(at):
    """Edge 4 at n_tau = 1 (the first build's headline setting) is a ~2% hop-rate
    deficit; the shorter window passes."""
    from paper_2004_09081_gb300 import workloads
    wl = workloads.batched_batio3(0)
    cells = [r.cells for r in wl.replicas]
    t = at.deficit_table()
    worst, e_min, est = at.batch_deficit(t, cells, 4, 1.0)
    assert e_min <= 4 and est["vacancies_only"][0] > 0.02 and not at.accepted(est, 0.01)
    worst, e_min, est = at.batch_deficit(t, cells, wl.edge, wl.n_tau)
    assert at.accepted(est, 0.01), (wl.edge, wl.n_tau, est)


def test_table_entry_reproduced_by_the_oracle(orc):
    """One stored per-seed deficit recomputed by the oracle, bit for bit (the
    table was written by oracle/window_deficit.py from the oracle alone)."""
    import json
    import os
    from oracle import window_deficit as wd
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2004_09081_gb300",
                        "window_deficit.json")
    stored = json.load(open(path))["table"]["4"]["vacancies_only"]["1.0"]["per_seed"][0]
    e, c, nt, s, hw, hb = wd._job((4, "vacancies_only", 1.0, 0))
    assert 1.0 - hw / hb == stored

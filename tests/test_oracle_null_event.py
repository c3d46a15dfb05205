"""Pins of the oracle's atom-based fragment kMC with null events (Sec. II.B,
Eqs. AtomP and TimeStepFrg), the atoms being the vacancies.

With one pick per step the method is the conventional kMC of Sec. II.A in
distribution: a pick of vacancy I with probability 1/N, then event i with
probability k_i/R_max, gives event i with probability k_i/sum k once the null
picks are discarded, and each non-null step advances the clock by an
exponential variate over the total rate.  Pinned by the single-vacancy closed
forms (never null, hop rate 8k, D = (2/3) k a^2) and by agreement with the
conventional BKL for D of V, O and H.  With many simultaneous picks the
reconciliation rule (a pick that shares a site with an earlier non-null pick
is null) must keep the lattice consistent even on crowded lattices.
"""
import math

import numpy as np
import pytest

KB = 8.617333262e-5
A = 1e13


def k_of(Ea, T):
    return A * math.exp(-Ea / (KB * T))


def test_pick_is_a_bijection_per_step():
    import oracle as orc
    for n in (1, 2, 5, 17, 64, 1000):
        perms = []
        for step in (0, 1, 7):
            p = [orc.null_pick(i, n, 3, 2, step) for i in range(n)]
            assert sorted(p) == list(range(n))
            perms.append(p)
        if n >= 5:
            assert perms[0] != perms[1] and perms[1] != perms[2] and perms[0] != perms[2]
    # the first pick of a step is uniform over the vacancies (chi-square, 16 dof)
    n, trials = 17, 6800
    cnt = np.bincount([orc.null_pick(0, n, 9, 0, st) for st in range(trials)], minlength=n)
    chi2 = float(((cnt - trials / n) ** 2 / (trials / n)).sum())
    assert chi2 < 40.0, chi2  # p ~ 1e-3


def test_pick_order_is_uniform_on_small_domains():
    """"Selected randomly" (Sec. II.B): on a small domain every one of the n!
    orders of the vacancies is equally likely from step to step (chi-square
    over all orders; a four-round network fails this for n >= 4)."""
    import oracle as orc
    for n, per in ((3, 400), (4, 100), (5, 40)):
        nf = math.factorial(n)
        steps = per * nf
        cnt = {}
        for st in range(steps):
            p = tuple(orc.null_pick(i, n, 5, 1, st) for i in range(n))
            cnt[p] = cnt.get(p, 0) + 1
        assert len(cnt) == nf
        c = np.array(list(cnt.values()), float)
        chi2 = float(((c - per) ** 2 / per).sum())
        dof = nf - 1
        assert chi2 < dof + 4.5 * math.sqrt(2 * dof), (n, chi2, dof)


def test_lone_vacancy_is_never_null_and_hops_at_8k(orc):
    """One vacancy: R_I = R_max, so every step executes exactly one hop, and
    the clock gives the hop rate 8k (Poisson count over many seeds)."""
    T, Ea, a = 800.0, 0.6, 3.905
    hops, tsum, r2 = 0, 0.0, []
    for seed in range(40):
        L = orc.Lattice((8, 8, 8), (2, 2, 2), 1, 0, seed=seed)
        L.set_rates(Ea, Ea, T, a_ang=a)
        L.null_run(1500, 1)
        c = L.counters()
        assert c["hops"] == 1500
        tt = L.null_clock()["t"]
        tsum += tt
        hops += c["hops"]
        d = L.records()[0, 2:5].astype(np.float64)
        r2.append((d**2).sum() * (0.5 * a * 1e-10) ** 2 / (6 * tt))
    # hop count fixed, clock random: total time ~ Gamma(hops, 8k)
    expect_t = hops / (8 * k_of(Ea, T))
    assert abs(tsum - expect_t) < 4 * expect_t / math.sqrt(hops)
    D_exact = 2.0 / 3.0 * k_of(Ea, T) * (a * 1e-10) ** 2
    r2 = np.array(r2)
    assert abs(r2.mean() - D_exact) < 3.5 * r2.std(ddof=1) / math.sqrt(len(r2)), r2.mean() / D_exact


def _D_all(L, t):
    out = []
    for sp in (0, 1, 2):
        m = L.moments(sp)
        out.append(m[4:7].sum() / max(m[0], 1) / (6 * t))
    return out


@pytest.mark.parametrize("n_frg", [1, 15])
def test_null_event_matches_conventional_bkl(orc, n_frg):
    """D of V, O and H from the null-event form (one pick per step: exact; one
    pick per vacancy: the fully parallel form) against the conventional BKL of
    Sec. II.A over the same simulated time (1% vacancies, x = 0.1 H-)."""
    T, cells, nv, nh = 800.0, (8, 8, 8), 15, 51
    res = {"null": [], "bkl": []}
    steps = 12000 if n_frg == 1 else 1200
    for seed in range(24):
        L = orc.Lattice(cells, (2, 2, 2), nv, nh, seed=seed, tracer=True)
        L.set_rates(0.6, 0.45, T)
        L.null_run(steps, n_frg)
        t = L.null_clock()["t"]
        res["null"].append(_D_all(L, t))
        B = orc.Lattice(cells, (2, 2, 2), nv, nh, seed=seed, tracer=True)
        B.set_rates(0.6, 0.45, T)
        B.bkl_run(t, stream=seed)
        res["bkl"].append(_D_all(B, t))
    a, b = np.array(res["null"]), np.array(res["bkl"])
    for sp in range(3):
        se = math.sqrt(a[:, sp].var(ddof=1) / len(a) + b[:, sp].var(ddof=1) / len(b))
        slack = 0.0 if n_frg == 1 else 0.05 * b[:, sp].mean()
        assert abs(a[:, sp].mean() - b[:, sp].mean()) < 3.5 * se + slack, (sp, a[:, sp].mean(), b[:, sp].mean(), se)


def test_crowded_parallel_picks_keep_the_lattice_consistent(orc):
    """30% vacancies, one pick per vacancy each step: picks collide often; after
    every step the lattice is consistent, each vacancy moved at most one
    neighbour step, and no more hops than picks happened."""
    nb = orc.neighbour_table()
    steps_ok = {tuple(v) for t in range(3) for v in nb[t, :, 4:7].tolist()}
    L = orc.Lattice((5, 5, 5), (1, 1, 1), 112, 40, seed=2, tracer=True)
    L.set_rates(0.6, 0.5, 900.0)
    occ0 = L.occupancy()
    prev = L.records()
    prev_by_id = {int(r[5]): r for r in prev}
    h0 = 0
    theta = 0.0
    for _ in range(60):
        L.null_run(1, 112)
        occ = L.occupancy()
        rec = L.records()
        assert np.array_equal(np.bincount(occ, minlength=3), np.bincount(occ0, minlength=3))
        assert set(rec[:, 1].tolist()) == set(np.flatnonzero(occ == 2).tolist())
        assert len(rec) == 112
        moved = 0
        for r in rec:
            d = tuple((r[2:5] - prev_by_id[int(r[5])][2:5]).tolist())
            assert d == (0, 0, 0) or d in steps_ok
            moved += d != (0, 0, 0)
        h = L.counters()["hops"]
        assert h - h0 == moved <= 112
        h0 = h
        th = L.null_clock()["theta"]
        assert th >= theta
        theta = th
        prev_by_id = {int(r[5]): r for r in rec}
        tr = L.tracer_field()
        assert np.array_equal(tr[occ != 2].sum(0) + rec[:, 2:5].sum(0), np.zeros(3))
    assert h0 > 500


def test_null_event_refuses_site_energies_and_bad_picks(orc):
    L = orc.Lattice((8, 8, 8), (2, 2, 2), 3, 0, seed=1)
    with pytest.raises(RuntimeError):
        L.null_run(1, 1)  # rates not set
    L.set_rates(0.6, 0.6, 800.0)
    with pytest.raises(RuntimeError):
        L.null_run(1, 0)
    L.set_site_energy(vv=[(2, 0.1)])
    with pytest.raises(RuntimeError):
        L.null_run(1, 1)

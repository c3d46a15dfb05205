"""Pins of the oracle's kMC against closed forms, invariants and the
conventional BKL algorithm (Sec. II.A of arXiv:2004.09081).

Closed forms for a single vacancy on the O sublattice (8 neighbours at
d = a/sqrt2, rate k each): hop rate 8k, D = Gamma d^2 / 6 = (2/3) k a^2.
Under a field along z with eps = q E a / (4 kB T):  v_z = (8/3) a k0 sinh(eps).
A single fragment makes the windowed scheme exact (the restart at each window
boundary is memoryless), so those pins are tight there; with several fragments
the synchronous-sublattice hand-off leaves an O(tau) deficit in the hop rate,
pinned by its bound and by its vanishing as tau -> 0.
"""
import math

import numpy as np
import pytest

KB = 8.617333262e-5
A = 1e13


def k_of(Ea, T):
    return A * math.exp(-Ea / (KB * T))


def walkers(orc, cells, nf, nv, seeds, Ea, T, windows, n_tau=1.0, Ez=0.0, a=3.905,
            precision=0):
    """Run `seeds` lattices; return per-vacancy displacements (a/2 units),
    total hops and simulated time."""
    disp, hops, t = [], 0, None
    for s in seeds:
        L = orc.Lattice(cells, nf, nv, 0, seed=s)
        L.set_rates(Ea, Ea, T, Ez=Ez, a_ang=a, n_tau=n_tau, precision=precision)
        L.run(windows)
        disp.append(L.records()[:, 2:5])
        hops += L.counters()["hops"]
        t = windows * L.params()["tau"]
    return np.concatenate(disp).astype(np.float64), hops, t


def test_conservation_and_record_consistency(orc):
    L = orc.Lattice((8, 8, 12), (2, 2, 4), 30, 100, seed=5, tracer=True)
    occ0 = L.occupancy()
    L.set_rates(0.6, 0.3, 700.0, Ez=3e7)
    for _ in range(5):
        L.run(40)
        occ = L.occupancy()
        assert np.array_equal(np.bincount(occ, minlength=3), np.bincount(occ0, minlength=3))
        rec = L.records()
        assert set(rec[:, 1].tolist()) == set(np.flatnonzero(occ == 2).tolist())
        assert len(rec) == 30 and sorted(rec[:, 5].tolist()) == list(range(30))
        # every record sits in the fragment that owns its site
        Lx, Ly, Lz = 8, 8, 12
        for f, s in rec[:, :2]:
            x, y, z = s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz
            assert f == ((z // 3) * 2 + y // 4) * 2 + x // 4
        # each exchange moves the vacancy by +d and the ion by -d: total is zero
        tr = L.tracer_field()
        ions = occ != 2
        assert np.array_equal(tr[ions].sum(0) + rec[:, 2:5].sum(0), np.zeros(3))
    assert L.counters()["hops"] > 200


def test_single_fragment_hop_rate_is_exact(orc):
    """One fragment: hops per vacancy per second = 8k (Poisson count)."""
    T, Ea = 800.0, 0.6
    _, hops, t = walkers(orc, (8, 8, 8), (1, 1, 1), 1, range(40), Ea, T, 2000)
    expect = 40 * 8 * k_of(Ea, T) * t
    assert abs(hops - expect) < 3.5 * math.sqrt(expect)


def test_single_vacancy_D_closed_form(orc):
    """D = Gamma d^2/6 with Gamma = 8k, d = a/sqrt2, for 1 and 2^3 fragments."""
    T, Ea, a = 800.0, 0.6, 3.905
    D_exact = 2.0 / 3.0 * k_of(Ea, T) * (a * 1e-10) ** 2
    h = 0.5 * a * 1e-10
    for nf in ((1, 1, 1), (2, 2, 2)):
        d, hops, t = walkers(orc, (12, 12, 12), nf, 8, range(60), Ea, T, 600, n_tau=0.5)
        r2 = (d**2).sum(1) * h * h / (6 * t)
        D, se = r2.mean(), r2.std(ddof=1) / math.sqrt(len(r2))
        bias = 0.0 if nf == (1, 1, 1) else 0.02 * D_exact  # O(tau) hand-off deficit
        assert abs(D - D_exact) < 3 * se + bias, (nf, D / D_exact, se / D_exact)
        # a wrong time convention (8 tau per window) would be off by 8x
        assert 0.8 < D / D_exact < 1.25


def test_single_vacancy_among_hydride_ions(orc):
    """The H- exchange rate, apart from the O one.  (1) Every other O site holds
    H-: all 8 exchanges of the vacancy take the H- barrier, so one fragment
    gives hop rate 8 k_H and D = (2/3) k_H a^2, whatever the (far higher) O
    barrier.  (2) A mixture: with equal barriers both ways the configurations
    of one vacancy among n_H H- and the rest O are equally likely at all
    times (the placement is uniform and the dynamics reversible with respect
    to the uniform measure), so the mean hop rate is exactly
    8 (p k_H + (1 - p) k_O) with p = n_H / (N - 1), N the O-sublattice sites."""
    T, a = 800.0, 3.905
    cells = (8, 8, 8)
    N = 3 * 8 ** 3
    h = 0.5 * a * 1e-10
    # (1) all H-
    Ea_O, Ea_H = 0.9, 0.6
    kH = k_of(Ea_H, T)
    disp, hops, t = [], 0, None
    for s in range(40):
        L = orc.Lattice(cells, (1, 1, 1), 1, N - 1, seed=s)
        L.set_rates(Ea_O, Ea_H, T, a_ang=a, n_tau=0.5)
        L.run(600)
        disp.append(L.records()[:, 2:5])
        hops += L.counters()["hops"]
        t = 600 * L.params()["tau"]
    expect = 40 * 8 * kH * t
    assert abs(hops - expect) < 3.5 * math.sqrt(expect), (hops, expect)
    d = np.concatenate(disp).astype(np.float64)
    r2 = (d ** 2).sum(1) * h * h / (6 * t)
    D_exact = 2.0 / 3.0 * kH * (a * 1e-10) ** 2
    D, se = r2.mean(), r2.std(ddof=1) / math.sqrt(len(r2))
    assert abs(D - D_exact) < 3 * se, (D / D_exact, se / D_exact)
    # (2) 30% of the other sites H-
    Ea_O, Ea_H = 0.6, 0.5
    kH, kO = k_of(Ea_H, T), k_of(Ea_O, T)
    nH = round(0.3 * (N - 1))
    p = nH / (N - 1)
    rates = []
    for s in range(48):
        L = orc.Lattice(cells, (1, 1, 1), 1, nH, seed=100 + s)
        L.set_rates(Ea_O, Ea_H, T, a_ang=a, n_tau=0.5)
        L.run(2000)
        rates.append(L.counters()["hops"] / (2000 * L.params()["tau"]))
    rates = np.array(rates)
    expect = 8 * (p * kH + (1 - p) * kO)
    m, se = rates.mean(), rates.std(ddof=1) / math.sqrt(len(rates))
    assert abs(m - expect) < 4 * se, (m / expect, se / expect)
    # the two plausible slips: every exchange at one barrier
    assert abs(m - 8 * kO) > 10 * se and abs(m - 8 * kH) > 10 * se


def test_windowing_error_vanishes_with_tau(orc):
    """Hop-rate deficit of the fragmented scheme is bounded by 4% x n_tau and
    shrinks as the window shortens (4^3 fragments of 4^3 cells)."""
    T, Ea = 800.0, 0.6
    k8 = 8 * k_of(Ea, T)
    defs = {}
    for n_tau in (0.25, 1.0, 2.0):
        _, hops, t = walkers(orc, (16, 16, 16), (4, 4, 4), 16, range(8), Ea, T,
                             int(300 / n_tau), n_tau=n_tau)
        defs[n_tau] = 1.0 - hops / (8 * 16 * k8 * t)  # 8 seeds x 16 vacancies
        se = 1 / math.sqrt(hops)
        assert -3 * se < defs[n_tau] < 0.04 * n_tau + 3 * se, (n_tau, defs[n_tau])
    assert defs[0.25] < defs[1.0] < defs[2.0]


def test_drift_under_field(orc):
    """v_z = (8/3) a k0 sinh(eps), eps = qEa/(4kT); zero field gives zero drift."""
    T, Ea, a, q = 800.0, 0.6, 3.905, 2.0
    eps = 0.4
    Ez = eps * 4 * KB * T / (q * a * 1e-10)
    k0 = k_of(Ea, T)
    h = 0.5 * a * 1e-10
    for field, v_exact in ((Ez, 8.0 / 3.0 * a * 1e-10 * k0 * math.sinh(eps)), (0.0, 0.0)):
        d, hops, t = walkers(orc, (8, 8, 8), (1, 1, 1), 1, range(300), Ea, T, 300, Ez=field, a=a)
        vz = d[:, 2] * h / t
        v, se = vz.mean(), vz.std(ddof=1) / math.sqrt(len(vz))
        assert abs(v - v_exact) < 3.5 * se, (v, v_exact, se)
    assert v_exact == 0.0


def test_drift_of_a_vacancy_among_hydride_ions(orc):
    """Every other O site holds H-, so every exchange moves charge +1 (H- <-> V)
    instead of the vacancy's +2: v_z = (8/3) a k_H sinh(eps_H), eps_H =
    E a / (4kT) with unit charge.  The field is the one that gives eps = 0.4
    for O exchanges; charge +2 here would double eps and the drift."""
    T, a = 800.0, 3.905
    N = 3 * 8 ** 3
    h = 0.5 * a * 1e-10
    Ez = 0.4 * 4 * KB * T / (2.0 * a * 1e-10)
    eps_H = 1.0 * Ez * a * 1e-10 / (4 * KB * T)
    v_exact = 8.0 / 3.0 * a * 1e-10 * k_of(0.6, T) * math.sinh(eps_H)
    vz = []
    for s in range(300):
        L = orc.Lattice((8, 8, 8), (1, 1, 1), 1, N - 1, seed=s)
        L.set_rates(0.9, 0.6, T, Ez=Ez, a_ang=a, n_tau=1.0)
        L.run(300)
        vz.append(L.records()[0, 4] * h / (300 * L.params()["tau"]))
    vz = np.array(vz, np.float64)
    v, se = vz.mean(), vz.std(ddof=1) / math.sqrt(len(vz))
    assert abs(v - v_exact) < 3.5 * se, (v / v_exact, se / v_exact)
    v_q2 = 8.0 / 3.0 * a * 1e-10 * k_of(0.6, T) * math.sinh(2 * eps_H)
    assert abs(v - v_q2) > 10 * se


def test_first_hop_is_uniform(orc):
    """Tiny lattice, one vacancy: the first exchange goes to each of the 8
    neighbours with probability 1/8 (all rates equal)."""
    tab = orc.neighbour_table()
    counts = np.zeros(8)
    n = 0
    for seed in range(1600):
        L = orc.Lattice((2, 2, 2), (1, 1, 1), 1, 0, seed=seed)
        t = int(L.records()[0, 1] // 8)  # site type of the vacancy
        L.set_rates(0.6, 0.6, 800.0, n_tau=0.2)
        for _ in range(200):
            L.run(1)
            if L.counters()["hops"]:
                break
        if L.counters()["hops"] != 1:
            continue
        d = tuple(L.records()[0, 2:5])
        counts[[tuple(tab[t, m, 4:7]) for m in range(8)].index(d)] += 1
        n += 1
    exp = n / 8
    assert n > 1200
    assert ((counts - exp) ** 2 / exp).sum() < 24  # df = 7, p ~ 1e-3


def test_vacancy_hydride_stationary_measure(orc):
    """One V and one H, symmetric exchange rates: the stationary measure is
    uniform, so P(V next to H) = 8/(N-1)."""
    N = 24
    adj = 0
    tab = orc.neighbour_table()
    trials = 2500
    for seed in range(trials):
        L = orc.Lattice((2, 2, 2), (1, 1, 1), 1, 1, seed=seed)
        L.set_rates(0.6, 0.5, 800.0)
        L.run(30)
        occ = L.occupancy()
        v = int(np.flatnonzero(occ == 2)[0])
        hsite = int(np.flatnonzero(occ == 1)[0])
        t, x, y, z = v // 8, v % 2, (v // 2) % 2, (v // 4) % 2
        for m in range(8):
            t2, dc = tab[t, m, 0], tab[t, m, 1:4]
            j = ((t2 * 2 + (z + dc[2]) % 2) * 2 + (y + dc[1]) % 2) * 2 + (x + dc[0]) % 2
            if j == hsite:
                adj += 1
                break
    p = 8 / (N - 1)
    assert abs(adj / trials - p) < 3.5 * math.sqrt(p * (1 - p) / trials)


def test_windowed_matches_conventional_bkl(orc):
    """Fragmented windowed kMC vs the conventional serial BKL of Sec. II.A on the
    same lattices: D of V, O and H agree (1% vacancies, x = 0.1 H-)."""
    T, cells, nv, nh = 800.0, (8, 8, 8), 15, 51
    res = {"win": {0: [], 1: [], 2: []}, "bkl": {0: [], 1: [], 2: []}}
    for seed in range(24):
        for kind in ("win", "bkl"):
            L = orc.Lattice(cells, (2, 2, 2), nv, nh, seed=seed, tracer=True)
            L.set_rates(0.6, 0.45, T, n_tau=0.5)
            W = 150
            t = W * L.params()["tau"]
            if kind == "win":
                L.run(W)
            else:
                L.bkl_run(t, stream=seed)
            for sp in (0, 1, 2):
                m = L.moments(sp)
                res[kind][sp].append(m[4:7].sum() / max(m[0], 1) / (6 * t))
    for sp in (0, 1, 2):
        a, b = np.array(res["win"][sp]), np.array(res["bkl"][sp])
        se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        assert abs(a.mean() - b.mean()) < 3.5 * se + 0.03 * b.mean(), (sp, a.mean(), b.mean(), se)


def test_fragment_count_invariance_like_table1(orc):
    """Table 1: D of the O vacancy does not depend on the number of fragments
    (spread of the means below one SD of the per-run estimates)."""
    import os
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                 "table1_fragment_invariance.txt"))
            if l.strip() and not l.startswith("#")]
    means = np.array([float(r[1]) for r in rows])
    sds = np.array([float(r[2]) for r in rows])
    assert means.max() - means.min() < sds.min()  # the paper's own statement
    T, Ea = 800.0, 0.6
    Ds, sd = [], []
    for nf in ((1, 1, 1), (2, 2, 2), (4, 4, 4)):
        d, _, t = walkers(orc, (16, 16, 16), nf, 12, range(12), Ea, T, 300, n_tau=0.5)
        r2 = (d**2).sum(1) / (6 * t)
        Ds.append(r2.mean())
        sd.append(r2.std(ddof=1) / math.sqrt(len(r2)))
    assert max(Ds) - min(Ds) < 3 * max(sd) + 0.02 * np.mean(Ds)


def test_arrhenius_slope_recovers_barrier(orc):
    """ln D vs 1/T over 300-700 K returns Ea within 5 meV."""
    Ea, a = 0.6, 3.905
    Ts = [300.0, 400.0, 500.0, 600.0, 700.0]
    lnD = []
    h = 0.5 * a * 1e-10
    for T in Ts:
        d, _, t = walkers(orc, (16, 16, 16), (1, 1, 1), 48, range(20), Ea, T, 150)
        lnD.append(math.log(((d**2).sum(1) * h * h).mean() / (6 * t)))
    slope = np.polyfit(1.0 / np.array(Ts), lnD, 1)[0]
    assert abs(-slope * KB - Ea) < 0.005, -slope * KB


def test_mixed_and_plain_agree(orc):
    """Same draws, fp32-quantised rates: the two forms follow the same
    trajectory until a rare rounding-induced divergence; D agrees to 1%."""
    occs = []
    for prec in (0, 1):
        L = orc.Lattice((16, 16, 16), (4, 4, 4), 60, 2400, seed=9, tracer=True)
        L.set_rates(0.7, 0.35, 600.0, precision=prec)
        L.run(1500)
        occs.append((L.occupancy(), L.counters()["hops"], L.diffusion(2)["D"]))
    (o0, h0, D0), (o1, h1, D1) = occs
    assert h0 > 10000
    assert abs(D0 - D1) <= 0.01 * D0
    assert abs(h0 - h1) <= 0.01 * h0


# ------------------------------------------------------------------ field: D tensor and drift
def _single_vacancy_chain(eps):
    """Exact long-time drift and D tensor of one vacancy under a z field, in
    units a = 1, k0 = 1, from the site-type Markov chain of the O sublattice
    (written from the geometry, not from the oracle): a type-t site hops by
    s_t e_t + s_u e_u (units a/2) to a type-u site, u != t, s = +-1, at rate
    exp(eps dz).  D_axis = sigma^2/2 with the asymptotic variance of an
    additive functional of a Markov chain, sigma^2 = sum_t pi_t sum_hops
    r (d + g(u) - g(t))^2, g solving Q g = -(b - vbar) (b: drift of type t)."""
    hops = {t: [] for t in range(3)}
    for t in range(3):
        for u in range(3):
            if u != t:
                for st in (-1, 1):
                    for su in (-1, 1):
                        d = np.zeros(3)
                        d[t], d[u] = st, su
                        hops[t].append((u, d, math.exp(eps * d[2])))
    Q, b = np.zeros((3, 3)), np.zeros((3, 3))
    for t in range(3):
        for u, d, r in hops[t]:
            Q[t, u] += r
            Q[t, t] -= r
            b[t] += r * d
    pi = np.linalg.lstsq(np.vstack([Q.T, np.ones(3)]), np.r_[0.0, 0.0, 0.0, 1.0], rcond=None)[0]
    vbar = pi @ b
    D = np.zeros(3)
    for ax in range(3):
        g = np.linalg.lstsq(np.vstack([Q, pi]), np.r_[-(b[:, ax] - vbar[ax]), 0.0], rcond=None)[0]
        s2 = sum(pi[t] * r * (d[ax] + g[u] - g[t]) ** 2 for t in range(3) for u, d, r in hops[t])
        D[ax] = s2 / 2 * 0.25          # (a/2)^2 per (unit displacement)^2
    return D, vbar * 0.5, pi


def test_single_vacancy_chain_reduces_to_closed_forms():
    """The exact chain reproduces the closed forms: D_xx = (1/3) a^2 k0 (1 +
    cosh eps) and v_z = (8/3) a k0 sinh eps exactly, D_zz = (2/3) a^2 k0 cosh eps
    to O(eps^2), D = (2/3) k a^2 at zero field, Einstein v = D qE/kT to O(eps^2)."""
    for eps in (0.0, 0.0582, 0.3, 1.0):
        D, v, pi = _single_vacancy_chain(eps)
        assert np.allclose(pi, 1 / 3)
        assert D[0] == pytest.approx((1 + math.cosh(eps)) / 3, rel=1e-12)
        assert D[1] == pytest.approx((1 + math.cosh(eps)) / 3, rel=1e-12)
        assert v[2] == pytest.approx(8 / 3 * math.sinh(eps), rel=1e-12, abs=1e-15)
        assert abs(D[2] / (2 / 3 * math.cosh(eps)) - 1) < 0.15 * eps * eps + 1e-12
        if eps:
            # qE/kT = 4 eps / a
            assert abs(v[2] / (D[2] * 4 * eps) - 1) < eps * eps


def _field_walkers(orc, eps, seeds, windows, nv=4, cells=(12, 12, 12), T=800.0, Ea=0.6, a=3.905, q=2.0):
    """Dilute vacancies under the field of strength eps = qEa/(4kT), one
    fragment (exact scheme).  Returns pooled moments, per-seed moments, t, Ez."""
    Ez = eps * 4 * KB * T / (q * a * 1e-10)
    pooled, per = np.zeros(7, np.int64), []
    t = None
    for s in seeds:
        L = orc.Lattice(cells, (1, 1, 1), nv, 0, seed=s)
        L.set_rates(Ea, Ea, T, Ez=Ez, a_ang=a, q_O=q)
        L.run(windows)
        m = L.moments(2)
        pooled += m
        per.append(m)
        t = windows * L.params()["tau"]
    return pooled, np.array(per), t, Ez


def test_field_D_tensor_and_drift(orc):
    """Strong field (eps = 1): the drift-corrected D_z of Sec. III's tracked
    trajectories against the exact chain value, D_xy against (1/3) a^2 k0 (1 +
    cosh eps), v_z against (8/3) a k0 sinh eps, each within 3 sigma of the
    spread over 384 independent lattices.  Without the drift correction D_z
    would be several times too large."""
    eps, T, Ea, a = 1.0, 800.0, 0.6, 3.905
    k0 = k_of(Ea, T)
    pooled, per, t, _ = _field_walkers(orc, eps, range(384), 700)
    d = orc.diffusion_from_moments(pooled, t, a)
    Dc, vc, _ = _single_vacancy_chain(eps)
    am = a * 1e-10
    D_exact = Dc * k0 * am * am
    v_exact = vc[2] * k0 * am
    h = 0.5 * am
    mu = pooled[3] / pooled[0]
    # per-lattice estimates about the pooled drift, for the spread
    n = per[:, 0].astype(float)
    varz = (per[:, 6] - 2 * mu * per[:, 3] + mu * mu * n) / n * h * h / (2 * t)
    dxy = (per[:, 4] + per[:, 5]) / n * h * h / (4 * t)
    vz = per[:, 3] / n * h / t
    se = lambda x: x.std(ddof=1) / math.sqrt(len(x))  # noqa: E731
    assert abs(d["D_z"] - D_exact[2]) < 3 * se(varz), (d["D_z"] / D_exact[2], se(varz) / D_exact[2])
    assert abs(d["D_xy"] - D_exact[0]) < 3 * se(dxy), (d["D_xy"] / D_exact[0], se(dxy) / D_exact[0])
    assert d["D_xy"] == pytest.approx(((1 + math.cosh(eps)) / 3) * k0 * am * am, rel=6 * se(dxy) / D_exact[0])
    assert abs(d["v"][2] - v_exact) < 3 * se(vz), (d["v"][2] / v_exact, se(vz) / v_exact)
    # the per-axis estimates of x and y carry no drift
    assert abs(d["v"][0]) < 3 * se(per[:, 1] / n * h / t) + 1e-30
    # the drift term is large here: <dz^2>/(2t) without it is far above D_z
    assert d["msd"][2] / (2 * t) > 3 * d["D_z"]
    # the zero-order form (2/3) a^2 k0 cosh eps is 6% low at eps = 1: the
    # measurement resolves the exact value from it
    assert D_exact[2] > 1.05 * (2 / 3) * math.cosh(eps) * k0 * am * am


def test_einstein_relation(orc):
    """Weak field (eps = 0.15): v_z = D_z qE/kT to O(eps^2) (Einstein), with the
    drift-corrected D_z measured on the same trajectories."""
    eps, T, a, q = 0.15, 800.0, 3.905, 2.0
    pooled, per, t, Ez = _field_walkers(orc, eps, range(384), 700)
    d = orc.diffusion_from_moments(pooled, t, a)
    ratio = d["v"][2] / (d["D_z"] * q * Ez / (KB * T))
    # relative spread of D_z over 1536 dilute vacancies (variance of a variance)
    rel = math.sqrt(2.0 / pooled[0])
    assert abs(ratio - 1) < 3 * rel + eps * eps / 3, (ratio, rel)

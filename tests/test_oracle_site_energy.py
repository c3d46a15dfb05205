"""Pins of the oracle's site-energy interactions.

The paper's dopant/defect section replaces the barrier Ea by Ea + dE_site/2,
with E_site a sum over coordination shells of vacancy-vacancy and
vacancy-dopant pair energies (its Table add01 lists the shell distances and
energies).  Every check here is computed independently of the oracle's own
shell tables and energy sums:

  * shell geometry    brute-force minimum-image distances over the whole lattice
                      and the textbook perovskite coordination numbers
  * single rates      one exponential A exp(-(Ea + dE/2)/(kB T)) with dE from a
                      brute-force pair sum over all vacancies and dopants
  * detailed balance  forward/backward rate ratio = exp(-dE_total/kT) with
                      E_total the brute-force configuration energy
  * stationary law    Boltzmann occupation of the shells around a dopant and of
                      the vacancy-pair shells (exact enumeration)
  * no partners       one vacancy with only V-V energies: the trajectory is
                      bit-identical to the one without interactions
"""
import math

import numpy as np
import pytest

import oracle as orc

KB = 8.617333262e-5
A = 1e13
# Table add01 of the paper, read on the ideal lattice (squared distance in
# (a/2)^2): V-V shells 2.76, 3.91, 4.78, 5.52, 6.17 A at a = 3.905 A; the
# V-Fe energies measured from the fourth shell (the non-interacting level).
PAPER_VV = [(2, 0.343), (4, 0.235), (6, 0.200), (8, 0.180), (10, 0.023)]
PAPER_VFE = [(1, 0.000 - 0.709), (5, 0.510 - 0.709), (9, 0.687 - 0.709)]


def positions(L):
    """Half-unit coordinates of all O sites (oracle site order) and B sites."""
    nx, ny, nz = L
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cell = np.stack([x.ravel(), y.ravel(), z.ravel()], 1) * 2
    o = np.concatenate([cell + np.eye(3, dtype=np.int64)[t] for t in range(3)])
    return o, cell


def min_image_d2(p, q, L):
    box = 2 * np.asarray(L)
    d = (p - q + box // 2) % box - box // 2
    return (d * d).sum(-1)


def brute_energy(occ, fe, L, vv, vfe, site, exclude=-1):
    """E_site in eV from pair distances over the whole lattice."""
    o, b = positions(L)
    E = 0.0
    vac = np.nonzero(occ == orc.SP_V)[0]
    vac = vac[(vac != site) & (vac != exclude)]
    d2 = min_image_d2(o[vac], o[site], L)
    for dd, e in vv:
        E += e * int((d2 == dd).sum())
    fes = np.nonzero(fe)[0]
    d2 = min_image_d2(b[fes], o[site], L)
    for dd, e in vfe:
        E += e * int((d2 == dd).sum())
    return E


def total_energy(occ, fe, L, vv, vfe):
    o, b = positions(L)
    vac = np.nonzero(occ == orc.SP_V)[0]
    E = 0.0
    for i, s in enumerate(vac):
        d2 = min_image_d2(o[vac[i + 1:]], o[s], L)
        for dd, e in vv:
            E += e * int((d2 == dd).sum())
        d2 = min_image_d2(b[np.nonzero(fe)[0]], o[s], L)
        for dd, e in vfe:
            E += e * int((d2 == dd).sum())
    return E


def test_shell_geometry_matches_brute_force():
    L = (7, 7, 7)
    lat = orc.Lattice(L, (1, 1, 1), 0, 0)
    vv = [(d, 0.01 * k) for k, d in enumerate((2, 4, 6, 8, 10, 12, 14, 16), 1)]
    fe = [(d, 0.01 * k) for k, d in enumerate((1, 5, 9, 13, 17), 1)]
    lat.set_site_energy(vv=vv, fe=fe)
    o, b = positions(L)
    for t in range(3):
        s = lat_site = (t * 7 + 3) * 49 + 3 * 7 + 3  # site of type t in cell (3,3,3)
        sh = lat.shells(t)
        got_vv = {}
        got_fe = {}
        for t2, dx, dy, dz, e in sh:
            key = int(e)
            tgt = got_fe if t2 < 0 else got_vv
            tgt[key] = tgt.get(key, 0) + 1
        d2o = min_image_d2(o, o[lat_site], L)
        d2b = min_image_d2(b, o[s], L)
        want_vv = {int(round(1e4 * e)): int((d2o == d).sum()) for d, e in vv}
        want_fe = {int(round(1e4 * e)): int((d2b == d).sum()) for d, e in fe}
        assert got_vv == want_vv
        assert got_fe == want_fe
    # textbook perovskite coordination: an O has 8 O at a/sqrt2 and 6 at a;
    # two B sites at a/2 (the linear B-O-B bridge) and 8 at sqrt5 a/2
    assert want_vv[100] == 8 and want_vv[200] == 6
    assert want_fe[100] == 2 and want_fe[200] == 8


def _random_config(L, n_vac, n_fe, n_h, seed):
    rng = np.random.default_rng(seed)
    nsite = 3 * L[0] * L[1] * L[2]
    ncell = L[0] * L[1] * L[2]
    occ = np.zeros(nsite, np.uint8)
    pick = rng.choice(nsite, n_vac + n_h, replace=False)
    occ[pick[:n_vac]] = orc.SP_V
    occ[pick[n_vac:]] = orc.SP_H
    fe = np.zeros(ncell, np.uint8)
    fe[rng.choice(ncell, n_fe, replace=False)] = 1
    return occ, fe


def _lattice(L, occ, fe, vv, vfe, T, nf=(1, 1, 1), Ea_O=0.6, Ea_H=0.3):
    lat = orc.Lattice(L, nf, 0, 0)
    lat.set_occupancy(occ)
    lat.set_dopants(fe)
    lat.set_site_energy(vv=vv, fe=vfe)
    lat.set_rates(Ea_O, Ea_H, T)
    return lat


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_event_rate_is_one_exponential(seed):
    L = (6, 6, 5)
    T = 700.0
    occ, fe = _random_config(L, 30, 12, 20, seed)
    lat = _lattice(L, occ, fe, PAPER_VV, PAPER_VFE, T)
    nb = orc.neighbour_table()
    n_checked = 0
    for s in np.nonzero(occ == orc.SP_V)[0]:
        t = s // (L[0] * L[1] * L[2])
        c = np.array(np.unravel_index(s % (L[0] * L[1] * L[2]), (L[2], L[1], L[0]))[::-1])
        for n in range(8):
            t2 = nb[t, n, 0]
            cj = (c + nb[t, n, 1:4]) % np.array(L)
            j = ((t2 * L[2] + cj[2]) * L[1] + cj[1]) * L[0] + cj[0]
            got = lat.event_rate(s, n)
            if occ[j] == orc.SP_V:
                assert got == 0.0
                continue
            Ea = 0.6 if occ[j] == orc.SP_O else 0.3
            dE = (brute_energy(occ, fe, L, PAPER_VV, PAPER_VFE, j, exclude=s)
                  - brute_energy(occ, fe, L, PAPER_VV, PAPER_VFE, s))
            want = A * math.exp(-(Ea + dE / 2) / (KB * T))
            assert got == pytest.approx(want, rel=1e-12), (s, n, dE)
            n_checked += 1
    assert n_checked > 100


def test_detailed_balance_against_total_energy():
    L = (6, 5, 6)
    T = 650.0
    occ, fe = _random_config(L, 25, 10, 0, 7)
    nb = orc.neighbour_table()
    ncell = L[0] * L[1] * L[2]
    rng = np.random.default_rng(5)
    checked = 0
    for s in rng.permutation(np.nonzero(occ == orc.SP_V)[0])[:12]:
        t = s // ncell
        c = np.array(np.unravel_index(s % ncell, (L[2], L[1], L[0]))[::-1])
        for n in range(8):
            t2 = nb[t, n, 0]
            cj = (c + nb[t, n, 1:4]) % np.array(L)
            j = ((t2 * L[2] + cj[2]) * L[1] + cj[1]) * L[0] + cj[0]
            if occ[j] == orc.SP_V:
                continue
            fwd = _lattice(L, occ, fe, PAPER_VV, PAPER_VFE, T).event_rate(s, n)
            occ2 = occ.copy()
            occ2[s], occ2[j] = occ[j], orc.SP_V
            back_n = [m for m in range(8)
                      if nb[t2, m, 0] == t and np.array_equal((cj + nb[t2, m, 1:4]) % np.array(L), c)]
            assert len(back_n) == 1
            bwd = _lattice(L, occ2, fe, PAPER_VV, PAPER_VFE, T).event_rate(j, back_n[0])
            dE = total_energy(occ2, fe, L, PAPER_VV, PAPER_VFE) - total_energy(occ, fe, L, PAPER_VV, PAPER_VFE)
            assert fwd / bwd == pytest.approx(math.exp(-dE / (KB * T)), rel=1e-11)
            checked += 1
    assert checked > 30


def test_lone_vacancy_with_vv_energies_is_bit_identical():
    """With one vacancy the V-V sum is empty: the factor is exactly 1."""
    runs = []
    for on in (False, True):
        lat = orc.Lattice((8, 8, 8), (2, 2, 2), 1, 0, seed=11)
        if on:
            lat.set_site_energy(vv=PAPER_VV)
        lat.set_rates(0.6, 0.3, 800.0)
        lat.run(300)
        runs.append((lat.occupancy(), lat.records(), lat.counters()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert runs[0][2]["hops"] > 150


def _sample_sites(lat, n_samples, burn=200):
    lat.run(burn)
    out = np.empty(n_samples, np.int64)
    for k in range(n_samples):
        lat.run(1)
        out[k] = lat.records()[0, 1]
    return out


def test_boltzmann_occupation_around_a_dopant():
    """1 vacancy + 1 dopant, one fragment (exact BKL): the time the vacancy
    spends at each site is the Boltzmann weight exp(-E/kT) (exact enumeration)."""
    L = (5, 5, 5)
    T = 800.0
    vfe = [(1, -0.30), (5, -0.15), (9, -0.05)]
    fe = np.zeros(125, np.uint8)
    fe[62] = 1
    occ = np.zeros(375, np.uint8)
    occ[0] = orc.SP_V
    lat = orc.Lattice(L, (1, 1, 1), 0, 0, seed=3)
    lat.set_occupancy(occ)
    lat.set_dopants(fe)
    lat.set_site_energy(fe=vfe)
    lat.set_rates(0.6, 0.3, T, n_tau=4.0)
    sites = _sample_sites(lat, 20000)
    o, b = positions(L)
    d2 = min_image_d2(o, b[62], L)
    E = np.zeros(375)
    for dd, e in vfe:
        E[d2 == dd] = e
    w = np.exp(-E / (KB * T))
    w /= w.sum()
    got = np.array([(d2[sites] == dd).mean() for dd, _ in vfe])
    want = np.array([w[d2 == dd].sum() for dd, _ in vfe])
    assert want[0] > 0.2  # the dopant traps: most weight in the first shell
    assert np.allclose(got, want, atol=0.03), (got, want)


def test_boltzmann_vacancy_pair_distribution():
    """2 vacancies with a V-V attraction, one fragment: pair-distance shells
    follow n_k exp(-e_k/kT) (exact enumeration over site pairs)."""
    L = (3, 3, 3)
    T = 600.0
    vv = [(2, -0.10), (4, -0.05)]
    occ = np.zeros(81, np.uint8)
    occ[0] = occ[50] = orc.SP_V
    lat = orc.Lattice(L, (1, 1, 1), 0, 0, seed=4)
    lat.set_occupancy(occ)
    lat.set_site_energy(vv=vv)
    lat.set_rates(0.6, 0.3, T, n_tau=4.0)
    lat.run(200)
    o, _ = positions(L)
    counts = np.zeros(3)
    n = 20000
    for _ in range(n):
        lat.run(1)
        r = lat.records()
        d2 = int(min_image_d2(o[r[0, 1]][None], o[r[1, 1]], L)[0])
        counts[0 if d2 == 2 else (1 if d2 == 4 else 2)] += 1
    # exact: over all ordered site pairs of distinct sites
    d2all = min_image_d2(o[:, None, :], o[None, :, :], L)
    np.fill_diagonal(d2all, -1)
    E = np.where(d2all == 2, -0.10, np.where(d2all == 4, -0.05, 0.0))
    w = np.exp(-E / (KB * T)) * (d2all >= 0)
    want = np.array([w[d2all == 2].sum(), w[d2all == 4].sum(), w[d2all > 4].sum()]) / w.sum()
    got = counts / n
    assert want[0] > 0.3  # the attraction binds the pair well above its 8/80 share
    assert np.allclose(got, want, atol=0.02), (got, want)


def test_site_energy_validation():
    # a lattice shorter than twice the reach would count a partner twice
    lat = orc.Lattice((4, 6, 6), (1, 1, 1), 1, 0)
    with pytest.raises(ValueError):
        lat.set_site_energy(vv=PAPER_VV)
    # same-colour fragments closer than 2 + reach would interact
    lat = orc.Lattice((12, 12, 12), (4, 4, 4), 1, 0)
    with pytest.raises(ValueError):
        lat.set_site_energy(vv=PAPER_VV)
    lat = orc.Lattice((16, 16, 16), (4, 4, 4), 1, 0)
    lat.set_site_energy(vv=PAPER_VV, fe=PAPER_VFE)
    with pytest.raises(ValueError):  # the mixed form has no site-energy rates
        lat.set_rates(0.6, 0.3, 800.0, precision=orc.MIXED)
    # a shell distance the O sublattice does not have
    lat = orc.Lattice((8, 8, 8), (1, 1, 1), 1, 0)
    with pytest.raises(ValueError):
        lat.set_site_energy(vv=[(3, 0.1)])


def test_dopant_placement_is_a_bijection_prefix():
    lat = orc.Lattice((9, 7, 5), (1, 1, 1), 3, 2, seed=9, n_Fe=40)
    d = lat.dopants()
    assert d.sum() == 40
    lat2 = orc.Lattice((9, 7, 5), (1, 1, 1), 3, 2, seed=9, n_Fe=41)
    # the first 40 cells of the permutation are shared
    assert np.all(lat2.dopants()[d == 1] == 1) and lat2.dopants().sum() == 41

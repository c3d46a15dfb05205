"""Pins of the electrostatics oracle (oracle/poisson.py and the frozen-field
term of the C oracle): the Poisson-solved potential of the paper's mu-scale
model, read with the vacancy charges as its source.

Checked independently of the FFT solve: the discrete equation by an explicit
7-point stencil, the continuum Coulomb law at a few lattice spacings, the
charge deposit's conservation, the cubic symmetry of a vacancy's own-potential
table, and detailed balance of the rates in a frozen potential.
"""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import poisson as ps

KB = 8.617333262e-5


def stencil(phi):
    out = 6.0 * phi
    for ax in range(3):
        out -= np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
    return out


def test_discrete_equation_and_zero_mean():
    rng = np.random.default_rng(1)
    L = (12, 10, 14)
    sites = rng.choice(3 * 12 * 10 * 14, 40, replace=False)
    Q = ps.node_charge(L, sites, q=2.0)
    assert abs(Q.sum()) < 1e-9
    # before the background each vacancy adds its whole charge
    assert np.isclose((Q - Q.min()).sum() + Q.min() * Q.size, 0.0)
    phi = ps.solve(Q, 4.01, 500.0)
    f = Q * ps.E_CHARGE / (ps.EPS0 * 500.0 * 4.01e-10)
    assert np.allclose(stencil(phi), f, rtol=0, atol=1e-12 * np.abs(f).max())
    assert abs(phi.mean()) < 1e-14 * np.abs(phi).max()


def test_point_charge_follows_coulomb():
    """A unit charge on one node: potential differences at a few spacings match
    e / (4 pi eps0 eps_r) (1/r1 - 1/r2) (the periodic images and the lattice
    shift both fade at r << L)."""
    n, c = 96, 48
    Q = np.zeros((n, n, n))
    Q[c, c, c] = 1.0
    Q -= Q.mean()
    a, er = 4.01, 100.0
    phi = ps.solve(Q, a, er)
    k = ps.E_CHARGE / (4 * math.pi * ps.EPS0 * er * a * 1e-10)
    ratio = []
    for r1, r2 in ((3, 6), (4, 8), (6, 12), (8, 16)):
        got = phi[c, c, c + r1] - phi[c, c, c + r2]
        ratio.append(got / (k * (1.0 / r1 - 1.0 / r2)))
    # the lattice correction fades as r grows; at 8..16 spacings it is gone
    assert ratio[0] > ratio[1] > ratio[2] > ratio[3]
    assert ratio[2] == pytest.approx(1.0, abs=0.015) and ratio[3] == pytest.approx(1.0, abs=0.005), ratio
    # isotropy of the discrete solution at r = 4 along the three axes
    assert phi[c, c, c + 4] == pytest.approx(phi[c, c + 4, c], rel=1e-12)
    assert phi[c, c, c + 4] == pytest.approx(phi[c + 4, c, c], rel=1e-12)


def test_self_table_is_one_negative_value():
    """An O site's deposit is symmetric under the three mirror planes through it
    and the swap of the two other axes, so all 8 hops (and all 3 site types)
    take the same share of the own potential; moving away lowers it."""
    nb = orc.neighbour_table()
    g = ps.self_table((16, 16, 16), 4.01, 50.0, nb)
    assert np.all(g == g[0, 0])
    assert g[0, 0] < 0


def test_frozen_field_rates_keep_detailed_balance():
    """In a frozen potential the hop rates satisfy k(s->j)/k(j->s) =
    exp(-(u(j) - u(s))/kT): the own-potential share cancels between the two
    directions, and the stationary measure is Boltzmann in u."""
    L = (8, 8, 8)
    T = 700.0
    rng = np.random.default_rng(3)
    occ = np.zeros(3 * 512, np.uint8)
    occ[rng.choice(3 * 512, 30, replace=False)] = 2
    nb = orc.neighbour_table()
    u = rng.integers(-3000, 3000, 3 * 512).astype(np.int32)
    g = np.full((3, 8), -250, np.int32)

    def lattice(o):
        lat = orc.Lattice(L, (1, 1, 1), 0, 0)
        lat.set_occupancy(o)
        lat.set_elec(u, g)
        lat.set_rates(0.6, 0.6, T)
        return lat

    checked = 0
    for s in np.flatnonzero(occ == 2)[:10]:
        t = s // 512
        c = np.array(np.unravel_index(s % 512, (8, 8, 8))[::-1])
        for n in range(8):
            t2 = nb[t, n, 0]
            cj = (c + nb[t, n, 1:4]) % 8
            j = ((t2 * 8 + cj[2]) * 8 + cj[1]) * 8 + cj[0]
            if occ[j] == 2:
                continue
            fwd = lattice(occ).event_rate(s, n)
            occ2 = occ.copy()
            occ2[s], occ2[j] = occ[j], 2
            back = [m for m in range(8) if nb[t2, m, 0] == t and np.array_equal((cj + nb[t2, m, 1:4]) % 8, c)]
            bwd = lattice(occ2).event_rate(j, back[0])
            dE = (int(u[j]) - int(u[s])) * 1e-4
            assert fwd / bwd == pytest.approx(math.exp(-dE / (KB * T)), rel=1e-11)
            # and one exponential with the own-potential share
            want = 1e13 * math.exp(-(0.6 + 0.5 * (dE - g[t, n] * 1e-4)) / (KB * T))
            assert fwd == pytest.approx(want, rel=1e-12)
            checked += 1
    assert checked > 30
    with pytest.raises(ValueError):
        lat = orc.Lattice(L, (1, 1, 1), 0, 0)
        lat.set_rates(0.6, 0.6, T, precision=orc.MIXED)
        lat.set_elec(u, g)

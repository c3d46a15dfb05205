"""Electrostatic potential of the vacancy charges -- oracle (TEST INFRASTRUCTURE).

The mu-scale model of the paper solves a Poisson equation for the
electrostatic potential (Sec. "Oxygen diffusion in mu-scale BaTiO3 model").
Reading taken here: the source is the vacancies' own charge, on the B-site
grid (one node per cell corner, spacing a, periodic in x, y and z), each
vacancy's charge q e split in halves between the two B nodes of its O site's
bond (site n + a/2 e_t between nodes n and n + e_t), against a uniform
neutralising background.  The discrete equation

    6 phi(n) - sum_{6 neighbours} phi(n') = Q(n) / (eps0 eps_r a)     [V]

is solved exactly by the discrete Fourier transform (eigenvalues
sum_d (2 - 2 cos(2 pi k_d / L_d)) of the 7-point operator), with the zero mode
(the background) removed.  The potential of an O site is the mean of its two
nodes.  Only the test-suite and the benchmark's CPU leg use this module.
"""
from __future__ import annotations

import numpy as np

E_CHARGE = 1.602176634e-19   # C
EPS0 = 8.8541878128e-12      # F/m


def node_charge(L, sites, q=2.0):
    """Q(n) in units of e on the B-site grid, array [z][y][x]: half of q at each
    end of every listed O site's bond, minus the mean."""
    nx, ny, nz = L
    ncell = nx * ny * nz
    Q = np.zeros(ncell)
    sites = np.asarray(sites, dtype=np.int64)
    t = sites // ncell
    c = sites % ncell
    x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
    np.add.at(Q, c, 0.5 * q)
    x2 = (x + (t == 0)) % nx
    y2 = (y + (t == 1)) % ny
    z2 = (z + (t == 2)) % nz
    np.add.at(Q, (z2 * ny + y2) * nx + x2, 0.5 * q)
    Q -= Q.mean()
    return Q.reshape(nz, ny, nx)


def solve(Q, a_ang, eps_r):
    """phi (V) of the discrete periodic Poisson equation for node charges Q (e)."""
    a = a_ang * 1e-10
    f = Q * E_CHARGE / (EPS0 * eps_r * a)
    nz, ny, nx = f.shape
    kz = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nz) / nz)
    ky = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(ny) / ny)
    kx = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nx) / nx)
    lam = kz[:, None, None] + ky[None, :, None] + kx[None, None, :]
    F = np.fft.fftn(f)
    lam[0, 0, 0] = 1.0
    P = F / lam
    P[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(P))


def site_potential(phi):
    """phi of every O site (site order of the lattice) from the node potentials:
    the mean of the two nodes of its bond."""
    nz, ny, nx = phi.shape
    out = []
    for axis in (2, 1, 0):  # t = 0 (x), 1 (y), 2 (z): neighbour node along that axis
        out.append(0.5 * (phi + np.roll(phi, -1, axis=axis)))
    return np.concatenate([o.ravel() for o in out])


def energy_units(phi_sites, q=2.0):
    """The vacancy's electrostatic energy q phi at every O site, rint(eV * 1e4)."""
    return np.rint(q * phi_sites * 1e4).astype(np.int64)


def self_table(L, a_ang, eps_r, nb_table, q=2.0):
    """g[t][n] = rint(q^2 (G(j, s) - G(s, s)) * 1e4) for a vacancy of type t and
    its neighbour n: the share of its own charge's potential that a hop takes
    along (G = potential per unit charge e of one vacancy's deposit, at O sites).
    Translation invariance makes it one table."""
    nx, ny, nz = L
    ncell = nx * ny * nz
    g = np.zeros((3, 8), np.int64)
    for t in range(3):
        s = t * ncell + ((nz // 2) * ny + ny // 2) * nx + nx // 2  # a site of type t, mid-lattice
        phi = solve(node_charge(L, [s], q=1.0), a_ang, eps_r)
        ps = site_potential(phi)
        c = np.array([nx // 2, ny // 2, nz // 2])
        for n in range(8):
            t2, dc = nb_table[t, n, 0], nb_table[t, n, 1:4]
            cj = (c + dc) % np.array(L)
            j = ((t2 * nz + cj[2]) * ny + cj[1]) * nx + cj[0]
            g[t, n] = int(np.rint(q * q * (ps[j] - ps[s]) * 1e4))
    return g

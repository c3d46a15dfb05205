"""Pins of the oracle's grain model (Sec. "Oxygen diffusion in mu-scale BaTiO3
model"): a periodic Voronoi tessellation of the cells, a boundary layer around
every grain boundary, and a barrier raised by 0.2 eV for hops that touch it.

Checked independently of the oracle: the grain map against a brute-force
nearest-seed search with seeds drawn from numpy's Philox, the boundary layer
against a neighbourhood scan, the boundary and bulk rates against their closed
forms, the symmetric barrier against the uniform stationary measure of one
vacancy, a zero barrier against the run without grains (bit-identical), and the
null-event form against the conventional BKL with grains.
"""
import math

import numpy as np
import pytest

KB = 8.617333262e-5
A = 1e13
M64 = (1 << 64) - 1


def numpy_block(ctr0, key):
    """Philox4x64-10 block of counter (ctr0, 0, 0, 0) from numpy's generator,
    which returns the block of its 256-bit counter + 1 first (so counter 0 is
    reached from all-ones)."""
    before = [ctr0 - 1, 0, 0, 0] if ctr0 > 0 else [M64, M64, M64, M64]
    bg = np.random.Philox(counter=np.array(before, np.uint64), key=np.array(key, np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def brute_grains(L, n_grains, seed, replica):
    key = [seed, (replica << 8) | 8]
    X = []
    for g in range(n_grains):
        y = numpy_block(g, key)
        X.append([(y[d] * 256 * L[d]) >> 64 for d in range(3)])
    X = np.array(X, np.int64)
    nx, ny, nz = L
    z, yy, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    C = np.stack([x.ravel(), yy.ravel(), z.ravel()], 1) * 256 + 128
    box = 256 * np.array(L, np.int64)
    d = np.abs(C[:, None, :] - X[None, :, :])
    d = np.minimum(d, box - d)
    d2 = (d * d).sum(-1)
    grain = d2.argmin(1)  # first minimum: ties go to the smaller seed index
    return grain


def brute_boundary(grain, L, width):
    g3 = grain.reshape(L[2], L[1], L[0])
    b = np.zeros_like(g3, dtype=bool)
    for dz in range(-width, width + 1):
        for dy in range(-width, width + 1):
            for dx in range(-width, width + 1):
                b |= np.roll(g3, (dz, dy, dx), axis=(0, 1, 2)) != g3
    return b.ravel().astype(np.uint8)


@pytest.mark.parametrize("L,G,width,seed", [((10, 8, 12), 7, 1, 3), ((9, 9, 9), 2, 2, 0), ((16, 6, 7), 4, 1, 5), ((24, 20, 16), 40, 1, 2)])
def test_grain_map_and_boundary_layer(orc, L, G, width, seed):
    lat = orc.Lattice(L, (1, 1, 1), 2, 0, seed=seed)
    lat.set_grains(G, width, 0.2)
    g, b = lat.grains()
    want = brute_grains(L, G, seed, 0)
    assert np.array_equal(g, want)
    assert np.array_equal(b, brute_boundary(want, L, width))
    assert 0 < b.sum() < b.size


def _cell_of(s, L):
    return s % (L[0] * L[1] * L[2])


def test_boundary_and_bulk_rates_closed_form(orc):
    L, T = (16, 16, 16), 700.0
    lat = orc.Lattice(L, (1, 1, 1), 60, 150, seed=2)
    lat.set_grains(4, 1, 0.2)
    lat.set_rates(0.7, 0.35, T, a_ang=4.01)
    _, bnd = lat.grains()
    occ = lat.occupancy()
    nb = orc.neighbour_table()
    seen = {0: 0, 1: 0}
    for s in np.flatnonzero(occ == 2):
        t = s // (L[0] * L[1] * L[2])
        c = np.array(np.unravel_index(_cell_of(s, L), (L[2], L[1], L[0]))[::-1])
        for n in range(8):
            cj = (c + nb[t, n, 1:4]) % np.array(L)
            j = ((nb[t, n, 0] * L[2] + cj[2]) * L[1] + cj[1]) * L[0] + cj[0]
            if occ[j] == 2:
                continue
            b = int(bnd[_cell_of(s, L)] or bnd[_cell_of(j, L)])
            Ea = (0.7 if occ[j] == 0 else 0.35) + 0.2 * b
            assert lat.event_rate(s, n) == pytest.approx(A * math.exp(-Ea / (KB * T)), rel=1e-13)
            seen[b] += 1
    assert seen[0] > 20 and seen[1] > 20


def test_zero_barrier_grains_are_bit_identical(orc):
    runs = []
    for grains in (False, True):
        lat = orc.Lattice((12, 12, 12), (2, 2, 2), 20, 50, seed=4, tracer=True)
        if grains:
            lat.set_grains(8, 1, 0.0)
        lat.set_rates(0.7, 0.35, 800.0, a_ang=4.01)
        lat.run(100)
        runs.append((lat.occupancy(), lat.records(), lat.tracer_field(), lat.counters()))
    for a, b in zip(runs[0][:3], runs[1][:3]):
        assert np.array_equal(a, b)
    assert runs[0][3] == runs[1][3]


def test_symmetric_barrier_keeps_the_uniform_measure(orc):
    """A raised barrier (not a site energy) leaves the stationary measure of one
    vacancy uniform: the time spent on boundary sites is their share."""
    L = (12, 12, 12)
    lat = orc.Lattice(L, (1, 1, 1), 1, 0, seed=1)
    lat.set_grains(2, 1, 0.15)
    lat.set_rates(0.6, 0.6, 900.0, n_tau=16.0)
    _, bnd = lat.grains()
    share = bnd.mean()
    assert 0.2 < share < 0.9
    lat.run(200)
    on = 0
    n = 20000
    for _ in range(n):
        lat.run(1)
        on += int(bnd[_cell_of(int(lat.records()[0, 1]), L)])
    # correlated samples: allow 5 standard errors of 2000 effective samples
    assert abs(on / n - share) < 5 * math.sqrt(share * (1 - share) / 2000), (on / n, share)


def test_grains_slow_the_vacancies_and_null_form_agrees_with_bkl(orc):
    T, cells, nv, nh = 800.0, (8, 8, 8), 15, 51
    D = {"none": [], "grains": []}
    res = {"null": [], "bkl": []}
    for seed in range(16):
        for kind in ("none", "grains"):
            L = orc.Lattice(cells, (2, 2, 2), nv, nh, seed=seed)
            if kind == "grains":
                L.set_grains(4, 1, 0.2)
            L.set_rates(0.6, 0.45, T)
            L.run(200)
            t = 200 * L.params()["tau"]
            m = L.moments(2)
            D[kind].append(m[4:7].sum() / max(m[0], 1) / (6 * t))
        N = orc.Lattice(cells, (2, 2, 2), nv, nh, seed=seed)
        N.set_grains(4, 1, 0.2)
        N.set_rates(0.6, 0.45, T)
        N.null_run(4000, 1)
        t = N.null_clock()["t"]
        m = N.moments(2)
        res["null"].append(m[4:7].sum() / max(m[0], 1) / (6 * t))
        B = orc.Lattice(cells, (2, 2, 2), nv, nh, seed=seed)
        B.set_grains(4, 1, 0.2)
        B.set_rates(0.6, 0.45, T)
        B.bkl_run(t, stream=seed)
        m = B.moments(2)
        res["bkl"].append(m[4:7].sum() / max(m[0], 1) / (6 * t))
    assert np.mean(D["grains"]) < 0.8 * np.mean(D["none"])
    a, b = np.array(res["null"]), np.array(res["bkl"])
    se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    assert abs(a.mean() - b.mean()) < 3.5 * se, (a.mean(), b.mean(), se)


def test_grain_validation(orc):
    lat = orc.Lattice((8, 8, 8), (1, 1, 1), 1, 0)
    with pytest.raises(ValueError):
        lat.set_grains(4, 0, 0.2)
    with pytest.raises(ValueError):
        lat.set_grains(4, 1, -0.1)
    with pytest.raises(ValueError):
        lat.set_grains(4, 4, 0.2)  # 8 cells < 2 x 4 + 1
    lat.set_grains(1, 1, 0.2)  # one grain: no boundaries, off
    g, b = lat.grains()
    assert b.sum() == 0

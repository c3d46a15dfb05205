"""Grains (Voronoi tessellation, boundary layer, raised boundary barrier) on the
GPU vs the CPU oracle, through the C ABI: the grain map and boundary layer,
and the trajectories of the colour-phase kernels (plain and mixed form), the
site-energy path and the null-event form with grains, bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_09081_gb300 import fkmc
    fkmc.load()
    return fkmc


def same(b, ref, r=0, tracer=False):
    assert np.array_equal(b.state(r), ref.occupancy())
    assert np.array_equal(b.records(r), ref.records())
    if tracer:
        assert np.array_equal(b.tracer_field(r), ref.tracer_field())
    assert b.info(r).hops == ref.counters()["hops"]


def test_grain_map_matches_oracle(fk, orc):
    cells = [(10, 8, 12), (16, 16, 16), (24, 20, 16)]
    b = fk.Batch([(*c, 4.01) for c in cells], [(5, 0)] * 3, 3, precision=1)
    for G, w in ((7, 1), (2, 2), (40, 1)):
        b.set_grains(G, w, 0.2)
        for r, c in enumerate(cells):
            ref = orc.Lattice(c, None, 5, 0, seed=3, replica=r, edge=4)
            assert tuple(b.info(r).nfrag) == ref.nf
            ref.set_grains(G, w, 0.2)
            g, bnd = b.grains(r)
            rg, rb = ref.grains()
            assert np.array_equal(g, rg)
            assert np.array_equal(bnd, rb)


@pytest.mark.parametrize("prec,small", [(0, -1), (0, 1), (1, -1), (1, 1), (1, 2)])
def test_grains_colour_phase_bit_exact(fk, orc, prec, small):
    cells, nf = (16, 12, 16), (4, 2, 4)
    b = fk.Batch([(*cells, 4.01)], [(40, 150)], 7, nfrag=nf, precision=prec, tracer=True, cap_v=64,
                 small_pass=small)
    b.set_grains(5, 1, 0.2)
    b.set_barriers(0.6, 0.5, 900.0, field_z=2e7)
    ref = orc.Lattice(cells, nf, 40, 150, seed=7, tracer=True)
    ref.set_grains(5, 1, 0.2)
    ref.set_rates(0.6, 0.5, 900.0, Ez=2e7, a_ang=4.01, cap_v=64, precision=prec)
    for _ in range(3):
        b.run(100)
        ref.run(100)
        same(b, ref, tracer=True)
    assert ref.counters()["hops"] > 600


def test_grains_with_site_energies_bit_exact(fk, orc):
    vv = [(2, 0.343), (4, 0.235), (6, 0.200), (8, 0.180), (10, 0.023)]
    fe = [(1, -0.709), (5, -0.199), (9, -0.022)]
    cells, nf = (16, 16, 16), (4, 4, 4)
    b = fk.Batch([(*cells, 3.905)], [(60, 0, 40)], 2, nfrag=nf, precision=0, cap_v=64)
    b.set_site_energy(vv, fe)
    b.set_barriers(0.6, 0.6, 900.0)
    b.set_grains(4, 1, 0.2)  # after the rates: tables rebuilt
    ref = orc.Lattice(cells, nf, 60, 0, seed=2, n_Fe=40)
    ref.set_site_energy(vv=vv, fe=fe)
    ref.set_rates(0.6, 0.6, 900.0, cap_v=64)
    ref.set_grains(4, 1, 0.2)
    for _ in range(2):
        b.run(30)
        ref.run(30)
        same(b, ref)


def test_grains_null_event_bit_exact(fk, orc):
    cells, nf = (12, 12, 12), (2, 2, 2)
    b = fk.Batch([(*cells, 3.905)], [(30, 120)], 5, nfrag=nf, precision=1, tracer=True, cap_v=64)
    b.set_barriers(0.6, 0.45, 800.0)
    b.set_grains(3, 1, 0.2)
    ref = orc.Lattice(cells, nf, 30, 120, seed=5, tracer=True)
    ref.set_rates(0.6, 0.45, 800.0, cap_v=64, precision=1)
    ref.set_grains(3, 1, 0.2)
    b.run_null(600, 30)
    ref.null_run(600, 30)
    same(b, ref, tracer=True)
    assert b.info().null_theta == ref.null_clock()["theta"]


def test_grains_off_again_and_resident_refused(fk, orc):
    b = fk.Batch([(8, 8, 8, 3.905)], [(15, 0)], 0, nfrag=(2, 2, 2), precision=1, cap_v=64)
    b.set_barriers(0.6, 0.6, 800.0)
    b.set_grains(3, 1, 0.2)
    b.set_grains(1)  # off: back to the bulk tables (and the resident kernel)
    ref = orc.Lattice((8, 8, 8), (2, 2, 2), 15, 0, seed=0)
    ref.set_rates(0.6, 0.6, 800.0, cap_v=64, precision=1)
    b.run(100)
    ref.run(100)
    same(b, ref)
    b2 = fk.Batch([(8, 8, 8, 3.905)], [(15, 0)], 0, nfrag=(2, 2, 2), precision=1, schedule=2)
    b2.set_barriers(0.6, 0.6, 800.0)
    with pytest.raises(fk.KmcError):
        b2.set_grains(3, 1, 0.2)  # the resident kernel has no grain tables
    with pytest.raises(fk.KmcError):
        b.set_grains(3, 4, 0.2)  # 8 cells < 2 x 4 + 1

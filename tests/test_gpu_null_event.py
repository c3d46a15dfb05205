"""The atom-based fragment kMC with null events (Sec. II.B, Eqs. AtomP and
TimeStepFrg) on the GPU vs the CPU oracle, through the C ABI.

Rates are exact integers, picks a keyed bijection, the reconciliation of
simultaneous picks an order-free rule, and the clock the same FP64 operations
on both sides: occupancy, records, tracer field, hop counts and the clock
must agree bit for bit.
"""
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


def pair(fk, orc, cells, nf, nv, nh, seed, T=800.0, Ea=(0.6, 0.45), tracer=True, prec=0, a=3.905, cap=64):
    b = fk.Batch([(*cells, a)], [(nv, nh)], seed, nfrag=nf, precision=prec, tracer=tracer, cap_v=cap)
    b.set_barriers(Ea[0], Ea[1], T)
    ref = orc.Lattice(cells, nf, nv, nh, seed=seed, tracer=tracer)
    ref.set_rates(Ea[0], Ea[1], T, a_ang=a, cap_v=cap, precision=prec)
    return b, ref


def same(b, ref, r=0, tracer=True):
    assert np.array_equal(b.state(r), ref.occupancy())
    assert np.array_equal(b.records(r), ref.records())
    if tracer:
        assert np.array_equal(b.tracer_field(r), ref.tracer_field())
    info, c, nc = b.info(r), ref.counters(), ref.null_clock()
    assert info.hops == c["hops"]
    assert info.null_steps == nc["steps"]
    assert info.null_theta == nc["theta"]  # the clock, bit for bit


@pytest.mark.parametrize("n_frg,steps", [(1, 3000), (4, 800), (15, 300), (1000, 300)])
def test_null_event_bit_exact(fk, orc, n_frg, steps):
    b, ref = pair(fk, orc, (8, 8, 8), (2, 2, 2), 15, 51, 3)
    for chunk in (steps // 3, steps - steps // 3):
        b.run_null(chunk, n_frg)
        ref.null_run(chunk, n_frg)
        same(b, ref)
    assert ref.counters()["hops"] > 100


def test_crowded_parallel_picks_bit_exact(fk, orc):
    """30% vacancies, one pick per vacancy: frequent collisions between picks."""
    b, ref = pair(fk, orc, (5, 5, 5), (1, 1, 1), 112, 40, 2, T=900.0, Ea=(0.6, 0.5), cap=128)
    for _ in range(3):
        b.run_null(20, 112)
        ref.null_run(20, 112)
        same(b, ref)


def test_batch_of_replicas(fk, orc):
    cells = [(12, 12, 12), (8, 10, 14), (16, 16, 16)]
    comps = [(40, 100), (25, 0), (90, 400)]
    T = [650.0, 800.0, 1000.0]
    b = fk.Batch([(*c, 4.01) for c in cells], comps, 11, edge=4, precision=1, tracer=True)
    b.set_barriers(0.7, 0.35, T)
    b.run_null(400, 30)
    for r in range(3):
        ref = orc.Lattice(cells[r], None, *comps[r], seed=11, replica=r, tracer=True, edge=4)
        assert tuple(b.info(r).nfrag) == ref.nf
        ref.set_rates(0.7, 0.35, T[r], a_ang=4.01, cap_v=b.info(r).cap_v, precision=1)
        ref.null_run(400, 30)
        same(b, ref, r)


@pytest.mark.parametrize("prec", [0, 1])
def test_alternating_with_the_spatial_scheme(fk, orc, prec):
    """Windows of the spatial scheme, then null-event steps, then windows again
    (records leave and re-enter their fragments)."""
    b, ref = pair(fk, orc, (8, 8, 12), (2, 2, 4), 30, 150, 7, T=700.0, prec=prec)
    b.run(40)
    ref.run(40)
    b.run_null(500, 10)
    ref.null_run(500, 10)
    same(b, ref)
    b.run(40)
    ref.run(40)
    same(b, ref)
    # D over the combined time: windows * tau + the null clock
    t_ref = ref.counters()["window"] * ref.params()["tau"] + ref.null_clock()["t"]
    assert b.info().null_time_s == pytest.approx(ref.null_clock()["t"], rel=1e-15)
    msd = b.D()[1] * 6 * t_ref
    assert msd > 0


def test_full_size_null_workload_sampled(fk, orc):
    """The benchmarked null-event lattice (BaTiO(3-x)H_x 128^3, 18,874 V, one
    pick per vacancy) after a few steps, bit for bit."""
    from paper_2004_09081_gb300 import workloads
    wl = workloads.null_batio3(0)
    rep = wl.replicas[0]
    b = fk.Batch([(*rep.cells, rep.a)], [(rep.n_vac, rep.n_H)], 0, nfrag=rep.nfrag, precision=wl.precision)
    b.set_barriers(rep.Ea_O, rep.Ea_H, rep.T)
    b.run_null(6, wl.notes["n_frg"])
    ref = orc.Lattice(rep.cells, rep.nfrag, rep.n_vac, rep.n_H, seed=0)
    ref.set_rates(rep.Ea_O, rep.Ea_H, rep.T, a_ang=rep.a, cap_v=b.info().cap_v, precision=wl.precision)
    ref.null_run(6, wl.notes["n_frg"])
    same(b, ref, tracer=False)
    assert ref.counters()["hops"] > 2000


def test_null_event_errors(fk):
    b = fk.Batch([(8, 8, 8, 3.905)], [(5, 0, 2)], 0, precision=0)
    with pytest.raises(fk.KmcError):
        b.run_null(1, 1)  # before the rates
    b.set_barriers(0.6, 0.6, 800.0)
    with pytest.raises(fk.KmcError):
        b.run_null(1, 0)
    b.set_site_energy([(2, 0.1)], [])
    with pytest.raises(fk.KmcError):
        b.run_null(1, 1)
    b.set_site_energy()
    b.run_null(3, 2)


def test_more_than_256_replicas_on_the_colour_phase_path(fk, orc):
    """300 replicas: the window set-up spans two blocks; every block must see
    the same window number."""
    n = 300
    b = fk.Batch([(8, 8, 8, 3.905)] * n, [(6, 10)] * n, 5, nfrag=(2, 2, 2), precision=0)
    b.set_barriers(0.6, 0.45, 800.0)
    b.run(12)
    for r in (0, 255, 256, 299):
        ref = orc.Lattice((8, 8, 8), (2, 2, 2), 6, 10, seed=5, replica=r)
        ref.set_rates(0.6, 0.45, 800.0, cap_v=b.info(r).cap_v)
        ref.run(12)
        assert np.array_equal(b.state(r), ref.occupancy())
        assert np.array_equal(b.records(r), ref.records())

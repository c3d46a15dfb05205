"""Site-energy interactions on the GPU vs the CPU oracle, through the C ABI.

The dopant/defect section of the paper shifts every barrier by half the
change of the vacancy's site energy (vacancy-vacancy and vacancy-dopant pair
energies by coordination shell, its Table add01).  The GPU keeps an integer
energy field of every O site, moved with each hop; the oracle sums the shells
from scratch for every event.  Both take the same integer energy differences
and the same FP64 products, so the plain form must agree bit for bit:
dopant placement, energy field, occupancy, records, tracer field, hop counts.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# Table add01 on the ideal lattice; V-Fe measured from the fourth shell
PAPER_VV = [(2, 0.343), (4, 0.235), (6, 0.200), (8, 0.180), (10, 0.023)]
PAPER_VFE = [(1, -0.709), (5, -0.199), (9, -0.022)]


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_09081_gb300 import fkmc
    fkmc.load()
    return fkmc


def oracle_field(ref):
    return np.array([ref.site_energy(s) for s in range(ref.nsite)], np.int64)


def make_pair(fk, orc, cells, nf, nv, nh, nfe, seed, T, vv=PAPER_VV, fe=PAPER_VFE, tracer=True, Ea=(0.6, 0.3),
              Ez=0.0, a=3.905, n_tau=1.0, cap=64):
    b = fk.Batch([(*cells, a)], [(nv, nh, nfe)], seed, nfrag=nf, precision=fk.FKMC_PLAIN, tracer=tracer,
                 cap_v=cap, n_tau=n_tau)
    b.set_site_energy(vv, fe)
    b.set_barriers(Ea[0], Ea[1], T, field_z=Ez)
    ref = orc.Lattice(cells, nf, nv, nh, seed=seed, tracer=tracer, n_Fe=nfe)
    ref.set_site_energy(vv=vv, fe=fe)
    ref.set_rates(Ea[0], Ea[1], T, Ez=Ez, a_ang=a, cap_v=cap, n_tau=n_tau)
    return b, ref


def check_equal(b, ref, tracer=True, field=True):
    assert np.array_equal(b.state(), ref.occupancy())
    assert np.array_equal(b.records(), ref.records())
    if tracer:
        assert np.array_equal(b.tracer_field(), ref.tracer_field())
    info, c = b.info(), ref.counters()
    assert (info.hops, info.handoffs, info.window) == (c["hops"], c["handoffs"], c["window"])
    if field:
        assert np.array_equal(b.site_field().astype(np.int64), oracle_field(ref))


def run_and_check(b, ref, windows, chunks=2, tracer=True):
    per = max(1, windows // chunks)
    done = 0
    while done < windows:
        w = min(per, windows - done)
        b.run(w)
        ref.run(w)
        done += w
        check_equal(b, ref, tracer=tracer)


def test_dopant_placement_bit_exact(fk, orc):
    for seed, cells, nfe in [(0, (16, 16, 16), 41), (5, (9, 7, 13), 100), (2, (5, 5, 5), 125)]:
        b = fk.Batch([(*cells, 3.905)], [(3, 0, nfe)], seed, precision=fk.FKMC_PLAIN)
        ref = orc.Lattice(cells, (1, 1, 1), 3, 0, seed=seed, n_Fe=nfe)
        assert np.array_equal(b.dopants(), ref.dopants())
        assert int(b.dopants().sum()) == nfe


def test_energy_field_matches_shell_sums(fk, orc):
    """The initial field (scattered from vacancies and dopants) equals the
    oracle's direct shell sums at every O site."""
    b, ref = make_pair(fk, orc, (12, 10, 14), (2, 2, 2), 60, 40, 30, 4, 800.0)
    assert np.array_equal(b.site_field().astype(np.int64), oracle_field(ref))


def test_interacting_srtio3_bit_exact(fk, orc):
    """16^3 cells, 4^3 fragments of edge 4 (the smallest edge the V-V reach
    allows), 1.2% vacancies, 1% Fe: field, occupancy and records after every
    chunk of windows."""
    b, ref = make_pair(fk, orc, (16, 16, 16), (4, 4, 4), 150, 0, 41, 1, 800.0, tracer=False)
    run_and_check(b, ref, 60, chunks=3, tracer=False)
    assert ref.counters()["hops"] > 3000


def test_interacting_hydride_tracer_bit_exact(fk, orc):
    b, ref = make_pair(fk, orc, (12, 12, 12), (2, 2, 2), 40, 200, 20, 3, 700.0)
    run_and_check(b, ref, 40)


def test_interacting_uneven_partition_bit_exact(fk, orc):
    b, ref = make_pair(fk, orc, (18, 13, 16), (4, 2, 4), 50, 80, 25, 9, 650.0, Ez=2e7)
    run_and_check(b, ref, 30)


def test_vv_only_and_fe_only(fk, orc):
    b, ref = make_pair(fk, orc, (10, 10, 10), (2, 2, 2), 40, 0, 0, 6, 900.0, fe=())
    run_and_check(b, ref, 40, tracer=True)
    b, ref = make_pair(fk, orc, (10, 10, 10), (2, 2, 2), 10, 0, 40, 7, 900.0, vv=())
    run_and_check(b, ref, 40, tracer=True)


def test_batch_of_interacting_replicas(fk, orc):
    # sizes whose even fragment counts at edge 4 keep every edge >= 4 (the V-V reach rule)
    cells = [(16, 16, 16), (8, 16, 24), (24, 8, 16)]
    comps = [(60, 0, 41), (30, 50, 20), (80, 0, 60)]
    T = [700.0, 850.0, 1000.0]
    b = fk.Batch([(*c, 4.01) for c in cells], comps, 13, edge=4, precision=fk.FKMC_PLAIN)
    b.set_site_energy(PAPER_VV, PAPER_VFE)
    b.set_barriers(0.7, 0.35, T)
    b.run(25)
    for r in range(3):
        ref = orc.Lattice(cells[r], None, comps[r][0], comps[r][1], seed=13, replica=r, n_Fe=comps[r][2], edge=4)
        assert tuple(b.info(r).nfrag) == ref.nf
        ref.set_site_energy(vv=PAPER_VV, fe=PAPER_VFE)
        ref.set_rates(0.7, 0.35, T[r], a_ang=4.01)
        ref.run(25)
        assert np.array_equal(b.state(r), ref.occupancy())
        assert np.array_equal(b.records(r), ref.records())
        assert np.array_equal(b.site_field(r).astype(np.int64), oracle_field(ref))


def test_explicit_state_and_dopants(fk, orc):
    """Written occupancy and dopant maps: the field is rebuilt, the run agrees."""
    cells = (10, 10, 10)
    rng = np.random.default_rng(3)
    occ = np.zeros(3000, np.uint8)
    pick = rng.choice(3000, 70, replace=False)
    occ[pick[:40]] = 2
    occ[pick[40:]] = 1
    fe = (rng.random(1000) < 0.03).astype(np.uint8)
    b, ref = make_pair(fk, orc, cells, (2, 2, 2), 0, 0, 0, 2, 750.0)
    b.write_state(occ)
    b.write_dopants(fe)
    ref.set_occupancy(occ)
    ref.set_dopants(fe)
    check_equal(b, ref)
    run_and_check(b, ref, 30)


def test_switching_interactions_off(fk, orc):
    b, _ = make_pair(fk, orc, (8, 8, 8), (2, 2, 2), 15, 0, 5, 0, 800.0, tracer=False)
    b.set_site_energy()  # off: back to the table rates
    ref = orc.Lattice((8, 8, 8), (2, 2, 2), 15, 0, seed=0, n_Fe=5)
    ref.set_rates(0.6, 0.3, 800.0)
    b.run(100)
    ref.run(100)
    assert np.array_equal(b.state(), ref.occupancy())
    assert np.array_equal(b.records(), ref.records())


def test_site_energy_errors(fk):
    b = fk.Batch([(12, 12, 12, 3.905)], [(5, 0, 3)], 0, edge=3, precision=fk.FKMC_PLAIN)
    with pytest.raises(fk.KmcError):  # edge 3 < 2 + V-V reach
        b.set_site_energy(PAPER_VV, PAPER_VFE)
    b.set_site_energy((), PAPER_VFE)  # dopant shells alone only need L >= 5
    b = fk.Batch([(16, 16, 16, 3.905)], [(5, 0, 3)], 0, edge=4, precision=fk.FKMC_MIXED)
    with pytest.raises(fk.KmcError):
        b.set_site_energy(PAPER_VV, PAPER_VFE)
    b = fk.Batch([(4, 8, 8, 3.905)], [(5, 0, 3)], 0, nfrag=(1, 2, 2), precision=fk.FKMC_PLAIN)
    with pytest.raises(fk.KmcError):  # 4 cells < 2 x reach + 1
        b.set_site_energy(PAPER_VV, ())


def test_full_size_fe_workload_sampled(fk, orc):
    """The benchmarked Fe-doped SrTiO3 batch (5 x 96^3 cells, 0.1% V, 0.1% Fe,
    600..1000 K) in the launch configuration the benchmark times; the coolest
    and the hottest replica checked bit for bit against the oracle."""
    from paper_2004_09081_gb300 import workloads
    wl = workloads.fe_srtio3(0)
    reps = wl.replicas
    b = fk.Batch([(*r.cells, r.a) for r in reps], [(r.n_vac, r.n_H, r.n_Fe) for r in reps], 0, edge=wl.edge,
                 precision=fk.FKMC_PLAIN)
    b.set_site_energy(wl.site["vv"], wl.site["fe"])
    b.set_barriers([r.Ea_O for r in reps], [r.Ea_H for r in reps], [r.T for r in reps])
    b.run(3)
    for r in (0, len(reps) - 1):
        rep = reps[r]
        ref = orc.Lattice(rep.cells, None, rep.n_vac, rep.n_H, seed=0, replica=r, n_Fe=rep.n_Fe, edge=wl.edge)
        assert tuple(b.info(r).nfrag) == ref.nf
        ref.set_site_energy(vv=wl.site["vv"], fe=wl.site["fe"])
        ref.set_rates(rep.Ea_O, rep.Ea_H, rep.T, a_ang=rep.a, cap_v=b.info(r).cap_v)
        ref.run(3)
        assert np.array_equal(b.dopants(r), ref.dopants())
        assert np.array_equal(b.state(r), ref.occupancy())
        assert np.array_equal(b.records(r), ref.records())
        assert b.info(r).hops == ref.counters()["hops"] > 0

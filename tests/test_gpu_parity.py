"""GPU path vs the CPU oracle through the C ABI.

The plain (FP64) and mixed (FP32 + u64 fixed point) forms must reproduce the
oracle's lattice bit for bit: occupancy, vacancy records (site, displacement,
id), tracer field and hop counts.  Both sides draw the same Philox streams and
take every floating-point decision with the same IEEE operations, so there is
nothing to tolerate.  Cases span several fragments per colour, several
32-event chunks per fragment, uneven and single-fragment partitions, batches
of uneven replicas, edge cases, and the full-size batched workload on sampled
replicas.
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


def run_pair(fk, orc, cells, nf, nv, nh, seed, windows, prec, tracer=True, T=800.0, Ea=(0.6, 0.3),
             Ez=0.0, a=3.905, cap=64, n_tau=1.0, chunks=1, schedule=0):
    sched, small, lane = form(schedule)
    b = fk.Batch([(*cells, a)], [(nv, nh)], seed, nfrag=nf, precision=prec, tracer=tracer, cap_v=cap,
                 n_tau=n_tau, schedule=sched, small_pass=small, lane_form=lane)
    b.set_barriers(Ea[0], Ea[1], T, field_z=Ez)
    ref = orc.Lattice(cells, nf, nv, nh, seed=seed, tracer=tracer)
    ref.set_rates(Ea[0], Ea[1], T, Ez=Ez, a_ang=a, cap_v=cap, n_tau=n_tau, precision=prec)
    # initial state
    assert np.array_equal(b.state(), ref.occupancy())
    assert np.array_equal(b.records(), ref.records())
    per = max(1, windows // chunks)
    done = 0
    while done < windows:
        w = min(per, windows - done)
        b.run(w)
        ref.run(w)
        done += w
        assert np.array_equal(b.state(), ref.occupancy()), f"occupancy differs after {done} windows"
        assert np.array_equal(b.records(), ref.records()), f"records differ after {done} windows"
        if tracer:
            assert np.array_equal(b.tracer_field(), ref.tracer_field())
        info, c = b.info(), ref.counters()
        assert (info.hops, info.handoffs, info.window) == (c["hops"], c["handoffs"], c["window"])
    return b, ref


# (precision, schedule): plain FP64 runs the colour-phase kernel; the mixed form
# runs both the colour-phase kernel (1) and the replica-resident kernel (2);
# 10 + s forces the small-fragment run pass beside the general one (plain:
# fragments with one or two vacancies, four or two per warp; mixed: one thread
# per fragment, in registers); 20 + s forces the grouped form in the mixed form
# too; 30 + s the persistent one-thread-per-fragment form
FORMS = [(0, 0), (1, 1), (1, 2), (0, 10), (1, 11), (1, 21), (1, 31)]


def form(sched):
    """schedule, small_pass and lane_form of a FORMS entry"""
    k, s = divmod(sched, 10)
    return {0: (s, -1, 0), 1: (s, 1, 1), 2: (s, 2, 0), 3: (s, 1, 2)}[k]


@pytest.mark.parametrize("prec,sched", FORMS)
def test_small_srtio3_bit_exact(fk, orc, prec, sched):
    """8^3 cells, 15 V, 2^3 fragments of 4^3 (one fragment per colour)."""
    b, ref = run_pair(fk, orc, (8, 8, 8), (2, 2, 2), 15, 0, 0, 600, prec, tracer=False, Ea=(0.6, 0.6),
                      chunks=3, schedule=sched)
    assert ref.counters()["hops"] > 5000


@pytest.mark.parametrize("prec,sched", FORMS)
def test_hydride_tracer_field_bit_exact(fk, orc, prec, sched):
    run_pair(fk, orc, (8, 8, 12), (2, 2, 4), 30, 150, 3, 150, prec, T=700.0, Ez=3e7, chunks=2, schedule=sched)


@pytest.mark.parametrize("prec,sched", FORMS)
def test_many_vacancies_per_fragment(fk, orc, prec, sched):
    """One fragment holding 60 vacancies: 15 chunks of 32 events, multi-pass
    scan and selection, periodic self-wrap."""
    run_pair(fk, orc, (8, 8, 8), (1, 1, 1), 60, 200, 7, 60, prec, cap=64, chunks=2, schedule=sched)


@pytest.mark.parametrize("nf", [(2, 4, 2), (1, 2, 4), (4, 1, 1)])
@pytest.mark.parametrize("prec,sched", FORMS)
def test_uneven_partitions(fk, orc, nf, prec, sched):
    run_pair(fk, orc, (10, 12, 9), nf, 25, 60, 11, 120, prec, Ez=-2e7, schedule=sched)


def test_srtio3_h_32c_plain(fk, orc):
    """32^3 cells, 492 V, 3277 H, 8^3 fragments (the T-sweep lattice at 500 K)."""
    run_pair(fk, orc, (32, 32, 32), (8, 8, 8), 492, 3277, 0, 30, 0, T=500.0, chunks=2)


def test_batch_of_uneven_replicas(fk, orc):
    """Replica r of a batch equals the oracle lattice keyed by (seed, r)."""
    cells = [(8, 8, 8), (12, 10, 8), (16, 16, 16), (9, 9, 9), (6, 8, 10)]
    comps = [(15, 0), (20, 40), (60, 300), (3, 10), (12, 30)]
    Ts = [800.0, 650.0, 500.0, 900.0, 1000.0]
    for prec, sched in FORMS:
        sc, sm, lf = form(sched)
        b = fk.Batch([(*c, 4.01) for c in cells], comps, 21, edge=4, precision=prec, tracer=True, cap_v=64,
                     schedule=sc, small_pass=sm, lane_form=lf)
        b.set_barriers(0.7, 0.35, Ts, field_z=[0, 1e7, 0, -1e7, 0])
        b.run(40)
        for r, (c, (nv, nh), T) in enumerate(zip(cells, comps, Ts)):
            info = b.info(r)
            ref = orc.Lattice(c, None, nv, nh, seed=21, replica=r, tracer=True, edge=4)
            assert tuple(info.nfrag) == ref.nf
            ref.set_rates(0.7, 0.35, T, Ez=[0, 1e7, 0, -1e7, 0][r], a_ang=4.01, cap_v=64, precision=prec)
            ref.run(40)
            assert np.array_equal(b.state(r), ref.occupancy()), r
            assert np.array_equal(b.records(r), ref.records()), r
            assert np.array_equal(b.tracer_field(r), ref.tracer_field()), r
            assert info.hops == ref.counters()["hops"]
            for sp in (0, 1, 2):
                assert np.array_equal(b.moments(r, sp), ref.moments(sp))


@pytest.mark.parametrize("sched", [1, 2])
def test_D_matches_oracle(fk, orc, sched):
    """K6 under a field: D = MSD/6t, D_xy, the drift-removed per-axis D (D_z
    along the field) and the drift velocity of every species, against the
    oracle's statement of the same from the same trajectories."""
    b, ref = run_pair(fk, orc, (12, 12, 12), (2, 2, 2), 40, 80, 5, 200, 1, T=900.0, Ez=1e8, schedule=sched)
    for sp in (0, 1, 2):
        Dx, D, Dxy, v = b.D(0, sp)
        d = ref.diffusion(sp)
        assert D == pytest.approx(d["D"], rel=1e-12)
        assert Dxy == pytest.approx(d["D_xy"], rel=1e-12)
        assert np.allclose(Dx, d["D_axes"], rtol=1e-12, atol=0)
        assert Dx[2] == pytest.approx(d["D_z"], rel=1e-12)
        assert np.allclose(v, d["v"], rtol=1e-12, atol=1e-30)
    # the field drives the vacancies along +z, and the drift is removed from D_z
    Dx, D, Dxy, v = b.D(0, fk.FKMC_V)
    assert v[2] > 0 and Dx[2] < b.moments(0, 2)[6] / 40 * (0.5 * 3.905e-10) ** 2 / (2 * ref.diffusion(2)["t"])


def test_edge_cases(fk, orc):
    for prec, sched in FORMS:
        # no vacancies: nothing moves, no hops
        b, _ = run_pair(fk, orc, (4, 4, 4), (2, 2, 2), 0, 10, 1, 5, prec, schedule=sched)
        assert b.info().hops == 0
        # every site a vacancy: no ion to exchange with
        b, _ = run_pair(fk, orc, (2, 2, 2), (1, 1, 1), 24, 0, 1, 5, prec, tracer=False, schedule=sched)
        assert b.info().hops == 0
        # a single vacancy on the smallest lattice, and degenerate 1-cell dimensions
        run_pair(fk, orc, (2, 2, 2), (1, 1, 1), 1, 3, 2, 300, prec, schedule=sched)
        run_pair(fk, orc, (1, 2, 3), (1, 1, 1), 2, 3, 2, 200, prec, schedule=sched)
        run_pair(fk, orc, (1, 1, 1), (1, 1, 1), 1, 1, 2, 200, prec, schedule=sched)


def test_explicit_state(fk, orc):
    """kmc_write_state: one vacancy at a chosen site next to an H."""
    cells, nf = (6, 6, 6), (2, 2, 2)
    occ = np.zeros(3 * 216, np.uint8)
    occ[5] = 2
    occ[216 + 5] = 1
    occ[400] = 2
    b = fk.Batch([(*cells, 3.905)], [(0, 0)], 4, nfrag=nf, tracer=True, cap_v=16)
    b.write_state(occ)
    b.set_barriers(0.6, 0.3, 700.0)
    ref = orc.Lattice(cells, nf, 0, 0, seed=4, tracer=True)
    ref.set_occupancy(occ)
    ref.set_rates(0.6, 0.3, 700.0, cap_v=16)
    assert np.array_equal(b.records(), ref.records())
    b.run(100)
    ref.run(100)
    assert np.array_equal(b.state(), ref.occupancy())
    assert np.array_equal(b.records(), ref.records())


def test_errors(fk):
    with pytest.raises(fk.KmcError) as e:
        fk.Batch([(8, 8, 8, 3.9)], [(0, 0)], 0, nfrag=(3, 2, 2))
    assert e.value.code == fk.FKMC_EINVAL
    with pytest.raises(fk.KmcError) as e:
        fk.Batch([(4, 4, 4, 3.9)], [(150, 0)], 0, nfrag=(2, 2, 2), cap_v=8)
    assert e.value.code == fk.FKMC_EOVERFLOW
    b = fk.Batch([(4, 4, 4, 3.9)], [(1, 0)], 0)
    with pytest.raises(fk.KmcError) as e:
        b.run(1)
    assert e.value.code == fk.FKMC_ESTATE
    with pytest.raises(fk.KmcError) as e:
        b.moments(0, fk.FKMC_O)
    assert e.value.code == fk.FKMC_ESTATE


def test_state_blob_roundtrip(fk):
    import torch
    b = fk.Batch([(8, 8, 8, 3.9), (6, 6, 6, 3.9)], [(10, 20), (5, 5)], 3)
    b.set_barriers(0.6, 0.3, 800.0)
    n = fk.kmc_state_bytes(b.h)
    host = torch.empty(n, dtype=torch.uint8).pin_memory()
    fk.kmc_download_state(b.h, host.data_ptr(), n)
    s0 = [b.state(0), b.state(1)]
    b.run(30)
    assert not np.array_equal(b.state(0), s0[0])
    fk.kmc_upload_state(b.h, host.data_ptr(), n)
    assert np.array_equal(b.state(0), s0[0]) and np.array_equal(b.state(1), s0[1])


def test_batched_workload_full_size_sampled(fk, orc):
    """The 256-replica batched workload in the benchmark's configuration:
    conservation on every replica, full bit-exact comparison on a sample."""
    from paper_2004_09081_gb300 import workloads
    wl = workloads.batched_batio3(0)
    reps = wl.replicas
    b = fk.Batch([(*r.cells, r.a) for r in reps], [(r.n_vac, r.n_H) for r in reps], 0, edge=wl.edge,
                 precision=wl.precision, n_tau=wl.n_tau, **wl.notes.get("launch_opts", {}))
    assert all(b.info(r).n_vac == reps[r].n_vac for r in range(len(reps)))
    b.set_barriers([r.Ea_O for r in reps], [r.Ea_H for r in reps], [r.T for r in reps])
    W = 8
    b.run(W)
    for r in range(len(reps)):
        m = b.moments(r, 2)
        assert m[0] == reps[r].n_vac
    cap = b.info(0).cap_v
    # the largest replicas (1024- or 512-thread class), a spread of others, and
    # one replica of every batch shape (phases, events) of the resident kernel's
    # first draws
    largest = sorted(range(len(reps)), key=lambda r: -reps[r].n_vac)[:3]
    by_draws = {}
    for r in range(len(reps)):
        if b.info(r).kernel == 1:
            by_draws.setdefault((b.info(r).draw_phases, b.info(r).draw_events), r)
    assert set(by_draws) <= {(8, 4), (4, 4), (2, 4), (8, 2), (4, 2), (2, 2), (1, 2)}
    assert (8, 4) in by_draws and any(ev == 2 for _, ev in by_draws)
    for r in sorted(set(largest) | {0, 1, 97, 200, 255} | set(by_draws.values())):
        rep = reps[r]
        info = b.info(r)
        ref = orc.Lattice(rep.cells, None, rep.n_vac, rep.n_H, seed=0, replica=r, edge=wl.edge)
        assert tuple(info.nfrag) == ref.nf
        ref.set_rates(rep.Ea_O, rep.Ea_H, rep.T, a_ang=rep.a, cap_v=cap, n_tau=wl.n_tau, precision=wl.precision)
        ref.run(W)
        occ = b.state(r)
        assert np.array_equal(np.bincount(occ, minlength=3)[1:], [rep.n_H, rep.n_vac])
        assert np.array_equal(occ, ref.occupancy()), r
        assert np.array_equal(b.records(r), ref.records()), r
        assert info.hops == ref.counters()["hops"]


def test_um_scale_full_size_properties(fk):
    """The 2500^3-cell BaTiO3 lattice under bias (4.7e10 O sites) in the
    benchmark's configuration.  Too large for the oracle, so it is held to
    properties valid at any size: every vacancy conserved, about one exchange
    per vacancy per window, and the drift velocity of the single-vacancy closed
    form v_z = (8/3) a k0 sinh(qEa/4kT) (within the windowing error)."""
    import math
    import torch
    from paper_2004_09081_gb300 import workloads
    free, _ = torch.cuda.mem_get_info()
    if free < 60 * 2**30:
        pytest.skip("needs ~40 GB of free device memory")
    wl = workloads.um_batio3_bias(0)
    rep = wl.replicas[0]
    b = fk.Batch([(*rep.cells, rep.a)], [(rep.n_vac, rep.n_H)], 0, edge=wl.edge, precision=wl.precision)
    b.set_barriers(rep.Ea_O, rep.Ea_H, rep.T, field_z=rep.field_z)
    s = b.run(2)
    m = b.moments()
    assert m[0] == rep.n_vac                      # every vacancy kept its record
    assert s.hops > 0.5 * rep.n_vac               # about one exchange per vacancy per window
    kB, q, a = 8.617333262e-5, 2.0, rep.a * 1e-10
    k0 = 1e13 * math.exp(-rep.Ea_O / (kB * rep.T))
    eps = q * rep.field_z * a / (4 * kB * rep.T)
    v_exact = 8.0 / 3.0 * a * k0 * math.sinh(eps)
    vz = b.D(0, fk.FKMC_V)[3][2]
    t = b.info().window * b.info().tau
    h = 0.5 * a
    var = (m[6] / m[0] - (m[3] / m[0]) ** 2) * h * h / t**2
    se = math.sqrt(var / m[0])
    assert abs(vz - v_exact) < 3 * se + 0.05 * v_exact, (vz, v_exact, se)
    b.close()


def test_cluster_pairs_bit_exact(fk, orc):
    """Large replicas run as 2-CTA thread-block clusters (state mirrored through
    distributed shared memory, half of each phase's fragments per CTA) give the
    oracle's lattice bit for bit."""
    cells = [(44, 44, 44), (40, 40, 42)]
    comps = [(2300, 9000), (1900, 4000)]
    Ts = [700.0, 900.0]
    b = fk.Batch([(*c, 4.01) for c in cells], comps, 13, edge=4, precision=1, cap_v=32, schedule=2,
                 cluster_top=2)
    b.set_barriers(0.7, 0.35, Ts)
    b.run(12)
    for r, (c, (nv, nh), T) in enumerate(zip(cells, comps, Ts)):
        info = b.info(r)
        ref = orc.Lattice(c, None, nv, nh, seed=13, replica=r, edge=4)
        assert tuple(info.nfrag) == ref.nf
        ref.set_rates(0.7, 0.35, T, a_ang=4.01, cap_v=32, precision=1)
        ref.run(12)
        assert info.hops == ref.counters()["hops"] > 0
        assert np.array_equal(b.state(r), ref.occupancy()), r
        assert np.array_equal(b.records(r), ref.records()), r


@pytest.mark.parametrize("prec,small,lane", [(0, 0, 0), (1, 0, 0), (1, 0, 2), (1, 2, 0)])
def test_small_pass_by_default_on_a_large_phase(fk, orc, prec, small, lane):
    """128^3 cells in 2^3-cell fragments: 32768 fragments per colour phase, so
    the small-fragment pass runs by default: beside the general one on a second
    stream inside the window graph (the plain form's grouped pass, the mixed
    form's one-thread-per-fragment pass in registers, or its grouped form on
    request), or in the mixed form's persistent form before it; bit for bit
    against the oracle."""
    cells, nf = (128, 128, 128), (64, 64, 64)
    nv = 3 * 128 ** 3 // 1000
    b = fk.Batch([(*cells, 4.01)], [(nv, 0)], 17, nfrag=nf, precision=prec, tracer=True, cap_v=16,
                 small_pass=small, lane_form=lane)
    b.set_barriers(0.7, 0.35, 600.0, field_z=1e7)
    ref = orc.Lattice(cells, nf, nv, 0, seed=17, tracer=True)
    ref.set_rates(0.7, 0.35, 600.0, Ez=1e7, a_ang=4.01, cap_v=16, precision=prec)
    s = b.run(8)
    # per window: set-up + 8 x (screen, small and general pass), or 8 x (the
    # persistent one-thread-per-fragment pass, general pass)
    assert s.launches == 8 * (17 if lane == 2 else 25)
    ref.run(8)
    assert np.array_equal(b.state(), ref.occupancy())
    assert np.array_equal(b.records(), ref.records())
    assert np.array_equal(b.tracer_field(), ref.tracer_field())
    info, c = b.info(), ref.counters()
    assert (info.hops, info.handoffs) == (c["hops"], c["handoffs"]) and c["hops"] > 30000


@pytest.mark.parametrize("small", [1, 2, 3])
def test_lane_pass_dense_fragments(fk, orc, small):
    """Mixed form, 8^3 cells in 64 fragments of 2^3 cells (24 O sites) with 200
    vacancies: fragments of every count from 1 to 7 (the register form takes
    up to 4, the persistent form up to 8, the rest go to the warp pass),
    neighbouring vacancies inside one fragment (their rates change with each
    other's hops), hand-offs every few events, H- and a field."""
    cells, nf = (8, 8, 8), (4, 4, 4)
    per_frag = np.bincount(orc.Lattice(cells, nf, 200, 300, seed=29).records()[:, 0], minlength=64)
    assert {1, 4, 5}.issubset(set(per_frag.tolist()))
    b, ref = run_pair(fk, orc, cells, nf, 200, 300, 29, 120, 1, T=750.0, Ez=2e7, cap=32, chunks=3,
                      schedule=10 * small + 1)
    assert ref.counters()["hops"] > 3000 and ref.counters()["handoffs"] > 1000


def test_persistent_lane_form_by_default_on_the_largest_phases(fk):
    """324^3 cells in 2^3-cell fragments: 531441 fragments per colour phase, at
    least the 2^19 from which the mixed form runs its persistent
    one-thread-per-fragment pass (two launches per phase); the register form on
    request takes the same trajectory (both are checked against the oracle on
    smaller lattices)."""
    cells, nf = (324, 324, 324), (162, 162, 162)
    nv = 3 * 324 ** 3 // 1000
    res = []
    for lane in (0, 1):
        b = fk.Batch([(*cells, 4.01)], [(nv, 0)], 5, nfrag=nf, precision=1, cap_v=16, lane_form=lane)
        b.set_barriers(0.7, 0.35, 600.0, field_z=1e7)
        s = b.run(2)
        assert s.launches == 2 * (17 if lane == 0 else 25)
        res.append((s.hops, b.info().handoffs, b.state(), b.records()))
        b.close()
    assert res[0][0] == res[1][0] > 0 and res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][3], res[1][3])


@pytest.mark.parametrize("cluster", [0, 2])
def test_resident_totals_carried_between_calls_and_dropped_on_change(fk, orc, cluster):
    """The resident kernels keep each fragment's exact event total from one call
    to the next; new rates (another temperature) or a rewritten state make them
    start over.  Runs split into calls, a rate change and a state round trip in
    between, bit for bit against the oracle doing the same."""
    cells, nf, nv, nh = (12, 12, 16), (2, 2, 4), 60, 150
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], 31, nfrag=nf, precision=1, cap_v=32, schedule=2,
                 cluster_ctas=cluster)
    ref = orc.Lattice(cells, nf, nv, nh, seed=31)
    b.set_barriers(0.6, 0.35, 900.0)
    ref.set_rates(0.6, 0.35, 900.0, a_ang=4.01, cap_v=32, precision=1)
    for w in (7, 1, 12):
        b.run(w)
        ref.run(w)
    assert np.array_equal(b.state(), ref.occupancy())
    b.set_barriers(0.6, 0.35, 1200.0)
    ref.set_rates(0.6, 0.35, 1200.0, a_ang=4.01, cap_v=32, precision=1)
    for w in (5, 9):
        b.run(w)
        ref.run(w)
    assert np.array_equal(b.state(), ref.occupancy())
    assert np.array_equal(b.records(), ref.records())
    # the same occupancy written back (records rebuilt from it: new ids, zero
    # displacements): the totals are recomputed and the occupancy goes on as the oracle's
    b.write_state(b.state())
    b.run(10)
    ref.run(10)
    assert np.array_equal(b.state(), ref.occupancy())
    assert b.info().hops == ref.counters()["hops"] > 200

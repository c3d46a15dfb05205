"""The cluster-resident kernel against the CPU oracle through the C ABI.

A replica too large for one SM's shared memory is held by a thread-block
cluster, one z-slab of fragment layers per CTA, with the neighbouring slabs'
sites, hand-offs (through the receiving CTA's inbox) and dirty marks reached
through distributed shared memory.  It must reproduce the oracle's lattice bit
for bit: occupancy, vacancy records, tracer field and hop counts.  Small
lattices are forced onto it (kmc_opts.cluster_ctas) with even and uneven slabs;
larger ones take it by default.
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


def check(b, ref, r=0, tracer=False):
    assert np.array_equal(b.state(r), ref.occupancy())
    assert np.array_equal(b.records(r), ref.records())
    if tracer:
        assert np.array_equal(b.tracer_field(r), ref.tracer_field())
    assert b.info(r).hops == ref.counters()["hops"]


@pytest.mark.parametrize("cells,nf,ncta", [((12, 12, 16), (2, 2, 4), 2), ((12, 12, 16), (2, 2, 4), 4),
                                           ((10, 12, 18), (2, 2, 6), 4), ((8, 10, 24), (2, 2, 8), 8)])
def test_forced_slabs_bit_exact(fk, orc, cells, nf, ncta):
    """Hydride, tracer and a field on 2 to 8 slabs (uneven: 6 layers on 4 CTAs);
    hand-offs across slab faces every few events."""
    nv, nh = 120, 200
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], 9, nfrag=nf, precision=1, tracer=True, cap_v=32, schedule=2,
                 cluster_ctas=ncta, n_tau=2.0)
    b.set_barriers(0.6, 0.4, 1000.0, field_z=3e7)
    ref = orc.Lattice(cells, nf, nv, nh, seed=9, tracer=True)
    ref.set_rates(0.6, 0.4, 1000.0, Ez=3e7, a_ang=4.01, cap_v=32, n_tau=2.0, precision=1)
    assert (b.info().kernel, b.info().ctas) == (2, ncta)
    for _ in range(3):
        s = b.run(40)
        assert s.launches == 1  # one cluster launch per call
        ref.run(40)
        check(b, ref, tracer=True)
    c = ref.counters()
    assert c["hops"] > 3000 and b.info().handoffs == c["handoffs"] > 600


def test_large_replica_takes_the_cluster_by_default(fk, orc):
    """64^3 cells in 4^3-cell fragments: the state (196 KB of occupancy alone)
    does not fit one SM, so the replica runs on a cluster by default; a batch
    beside it with a small replica on the single-CTA kernel."""
    cells = [(64, 64, 64), (12, 12, 12)]
    comps = [(2000, 6000), (20, 50)]
    b = fk.Batch([(*c, 4.01) for c in cells], comps, 4, edge=4, precision=1, cap_v=32)
    b.set_barriers(0.7, 0.35, [600.0, 900.0], field_z=[1e7, 0.0])
    assert b.info(0).kernel == 2 and b.info(1).kernel == 1 and b.info(1).ctas == 1
    s = b.run(12)
    assert s.launches == 2  # the cluster launch and the single-CTA class launch
    for r, (c, (nv, nh)) in enumerate(zip(cells, comps)):
        ref = orc.Lattice(c, None, nv, nh, seed=4, replica=r, edge=4)
        ref.set_rates(0.7, 0.35, [600.0, 900.0][r], Ez=[1e7, 0.0][r], a_ang=4.01, cap_v=32, precision=1)
        ref.run(12)
        check(b, ref, r)
        assert ref.counters()["hops"] > 0


def test_bulk_hydride_lattice_on_sixteen_slabs(fk, orc):
    """The 128^3 BaTiO(3-x)H_x lattice (x = 0.05, 0.3% V, 400 K, 16^3 fragments
    of 8^3 cells): one fragment layer per CTA of a 16-CTA cluster."""
    cells, nf = (128, 128, 128), (16, 16, 16)
    nv, nh = 18874, 104858
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], 0, nfrag=nf, precision=1, n_tau=0.5)
    b.set_barriers(0.7, 0.35, 400.0)
    ref = orc.Lattice(cells, nf, nv, nh, seed=0)
    ref.set_rates(0.7, 0.35, 400.0, a_ang=4.01, cap_v=b.info().cap_v, n_tau=0.5, precision=1)
    assert (b.info().kernel, b.info().ctas) == (2, 16)
    s = b.run(24)
    assert s.launches == 1
    ref.run(24)
    check(b, ref)
    assert ref.counters()["hops"] > 100

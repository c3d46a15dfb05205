"""Checkpoint / resume and failure detection through the C ABI.

Resume: a batch saved with kmc_download_state and loaded into a fresh batch
of the same shape continues bit for bit as the unbroken run -- occupancy,
records, tracer field, hop and hand-off counters, window counter and the
null-event clock -- because every random stream is keyed by counters the
blob carries.  Failure detection, without faulting the GPU: the resident
kernel's bounded wait on a barrier that nothing completes gives up and
kmc_run reports FKMC_ETIMEOUT with the state untouched and the context
usable; an allocator that starts returning NULL gives FKMC_ENOMEM and leaves
the batch usable.
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


def snapshot(b):
    """Everything observable about a batch, replica by replica."""
    out = []
    for r in range(b.n):
        info = b.info(r)
        row = {"occ": b.state(r), "rec": b.records(r), "hops": info.hops, "hand": info.handoffs,
               "window": info.window, "null_steps": info.null_steps, "null_theta": info.null_theta}
        if b._opts.tracer:
            row["tracer"] = b.tracer_field(r)
        out.append(row)
    return out


def same(a, b):
    assert len(a) == len(b)
    for ra, rb in zip(a, b):
        assert ra.keys() == rb.keys()
        for k in ra:
            if isinstance(ra[k], np.ndarray):
                assert np.array_equal(ra[k], rb[k]), k
            else:
                assert ra[k] == rb[k], k


def blob(fk, b):
    import torch
    n = fk.kmc_state_bytes(b.h)
    host = torch.empty(n, dtype=torch.uint8).pin_memory()
    fk.kmc_download_state(b.h, host.data_ptr(), n)
    return host


CELLS = [(12, 12, 12), (16, 12, 8), (10, 10, 10)]
COMPS = [(30, 90), (25, 40), (12, 0)]
TS = [700.0, 900.0, 1000.0]


def make(fk, prec, sched, tracer=True, seed=5):
    b = fk.Batch([(*c, 4.01) for c in CELLS], COMPS, seed, edge=4, precision=prec, tracer=tracer, cap_v=32,
                 schedule=sched)
    b.set_barriers(0.7, 0.35, TS, field_z=[0.0, 2e7, -1e7])
    return b


@pytest.mark.parametrize("prec,sched", [(0, 0), (1, 1), (1, 2)])
def test_resume_is_bit_exact(fk, prec, sched):
    """save after 30 windows and 40 null-event steps; the unbroken run and a
    fresh batch loaded from the blob then run 25 windows and 30 steps alike."""
    a = make(fk, prec, sched)
    a.run(30)
    a.run_null(40, 6)
    saved = blob(fk, a)
    a.run(25)
    a.run_null(30, 6)
    a.run(5)
    b = make(fk, prec, sched)
    b.run(3)  # a different state, overwritten by the upload
    fk.kmc_upload_state(b.h, saved.data_ptr(), saved.numel())
    b.run(25)
    b.run_null(30, 6)
    b.run(5)
    same(snapshot(a), snapshot(b))
    for r in range(a.n):
        for sp in (0, 1, 2):
            assert np.array_equal(a.moments(r, sp), b.moments(r, sp))


def test_resume_with_site_energy_and_electrostatics(fk):
    """Plain form with V-V / V-Fe shells and the Poisson-solved potential
    (refreshed every 4 windows, warm-started): the blob carries the dopants,
    the energies u, the warm-start potential and the windows since the solve."""
    cells, comps = [(16, 16, 16)], [(40, 0, 30)]

    def mk():
        b = fk.Batch([(*c, 3.905) for c in cells], comps, 9, edge=4, precision=0, tracer=True)
        b.set_site_energy([(2, 0.343), (4, 0.235)], [(1, -0.709), (5, -0.199)])
        b.set_barriers(0.6, 0.3, 900.0, field_z=1e7)
        b.set_electrostatics(eps_r=1000.0, refresh_windows=4, cycles=12, warm_cycles=6)
        return b

    a = mk()
    a.run(10)  # 10 windows: the blob is taken 2 windows after a refresh
    saved = blob(fk, a)
    a.run(13)
    b = mk()
    fk.kmc_upload_state(b.h, saved.data_ptr(), saved.numel())
    b.run(13)
    same(snapshot(a), snapshot(b))
    assert np.array_equal(a.site_field(), b.site_field())
    assert np.array_equal(a.potential_energy()[0], b.potential_energy()[0])


def test_blob_of_another_shape_is_rejected(fk):
    a = make(fk, 1, 1, tracer=True)
    saved = blob(fk, a)
    b = make(fk, 1, 1, tracer=False)
    with pytest.raises(fk.KmcError) as e:
        fk.kmc_upload_state(b.h, saved.data_ptr(), saved.numel())
    assert e.value.code == fk.FKMC_EINVAL
    bad = saved.clone().pin_memory()
    bad[0] ^= 1  # the magic word
    with pytest.raises(fk.KmcError) as e:
        fk.kmc_upload_state(a.h, bad.data_ptr(), bad.numel())
    assert e.value.code == fk.FKMC_EINVAL


def test_bounded_wait_times_out_and_context_survives(fk, orc):
    """The resident kernel waits on a barrier that nothing completes, gives up
    after 2 ms and reports it: FKMC_ETIMEOUT, no window run, state untouched.
    The context stays usable: a batch without the test wait then matches the
    oracle bit for bit."""
    cells, nv, nh = (12, 12, 12), 20, 60
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], 3, edge=4, precision=1, cap_v=32, schedule=2,
                 test_stuck_wait_us=2000)
    b.set_barriers(0.7, 0.35, 800.0)
    occ0, rec0 = b.state(), b.records()
    with pytest.raises(fk.KmcError) as e:
        b.run(5)
    assert e.value.code == fk.FKMC_ETIMEOUT
    assert np.array_equal(b.state(), occ0) and np.array_equal(b.records(), rec0)
    assert b.info().hops == 0
    ok = fk.Batch([(*cells, 4.01)], [(nv, nh)], 3, edge=4, precision=1, cap_v=32, schedule=2)
    ok.set_barriers(0.7, 0.35, 800.0)
    ok.run(20)
    ref = orc.Lattice(cells, None, nv, nh, seed=3, edge=4)
    ref.set_rates(0.7, 0.35, 800.0, a_ang=4.01, cap_v=32, precision=1)
    ref.run(20)
    assert np.array_equal(ok.state(), ref.occupancy())
    assert ok.info().hops == ref.counters()["hops"] > 0


class FailingAllocator:
    """Torch memory through the ABI's callback, until told to fail."""

    def __init__(self, fk):
        self.inner = fk.TorchAllocator()
        self.fail = False
        self.c_alloc = fk.kmc_alloc_fn(self._alloc)
        self.c_free = self.inner.c_free

    def _alloc(self, ctx, n):
        return None if self.fail else self.inner._alloc(ctx, n)


def test_enomem_after_creation_leaves_the_batch_usable(fk, orc):
    al = FailingAllocator(fk)
    b = fk.Batch([(12, 12, 12, 4.01)], [(20, 40)], 8, edge=4, precision=1, cap_v=32, alloc=al)
    b.set_barriers(0.7, 0.35, 800.0)
    al.fail = True
    for call in (lambda: b.run_null(5, 4), lambda: b.set_grains(4, 1, 0.2)):
        with pytest.raises(fk.KmcError) as e:
            call()
        assert e.value.code == fk.FKMC_ENOMEM
    al.fail = False
    b.set_grains(0)  # nothing was set
    b.run(15)
    ref = orc.Lattice((12, 12, 12), None, 20, 40, seed=8, edge=4)
    ref.set_rates(0.7, 0.35, 800.0, a_ang=4.01, cap_v=32, precision=1)
    ref.run(15)
    assert np.array_equal(b.state(), ref.occupancy())
    assert b.info().hops == ref.counters()["hops"]

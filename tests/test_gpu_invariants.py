"""Invariant check of the device state (kmc_check_invariants) through the C ABI.

Every event exchanges a vacancy with a neighbouring ion (Sec. II.A), so the
vacancy and H- counts never change, and the vacancy records must describe the
occupancy: one record per vacancy site, listed by the fragment owning it.
After every window of runs through each kernel family -- the replica-resident
kernel, the cluster-resident kernel (forced slabs), the colour-phase kernels
(plain form, small-fragment pass forced) and the null-event form -- the
check's census equals that of the oracle's occupancy, its hash sums equal
sums computed here from the oracle's vacancy sites, records and ids, and it
reports ok.  Corrupted states uploaded as a state blob (a vacancy cleared in
the occupancy, a record id changed, a fragment count beyond cap_v) are
reported; nothing is run on them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = np.uint64


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_09081_gb300 import fkmc
    fkmc.load()
    return fkmc


def mix64(z):
    """SplitMix64's output step: Weyl increment, then the xor-shift-multiply
    finaliser (Stafford's Mix13 constants), on uint64 with wrap-around."""
    z = np.asarray(z, dtype=np.uint64) + M(0x9E3779B97F4A7C15)
    z = (z ^ (z >> M(30))) * M(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> M(27))) * M(0x94D049BB133111EB)
    return z ^ (z >> M(31))


def hsum(values) -> int:
    return int(np.sum(mix64(values), dtype=np.uint64)) if len(values) else 0


def check_against_oracle(fk, b, ref, nv, nh):
    inv = b.check()
    occ = ref.occupancy()
    census = np.bincount(occ, minlength=4)
    assert list(inv.sites) == list(census[:4])
    assert (inv.sites[fk.FKMC_V], inv.sites[fk.FKMC_H], inv.sites[3]) == (nv, nh, 0)
    rec = ref.records()  # rows {fragment, site, dx, dy, dz, id}
    assert inv.records == len(rec) == nv
    assert (inv.rec_not_vacancy, inv.rec_wrong_fragment, inv.rec_outside, inv.frag_bad_count) == (0, 0, 0, 0)
    assert inv.hash_vac_sites == hsum(np.nonzero(occ == fk.FKMC_V)[0])
    assert inv.hash_rec_sites == hsum(rec[:, 1])
    assert inv.hash_rec_ids == inv.hash_ids_expected == hsum(np.arange(nv))
    assert inv.ok == 1


@pytest.mark.parametrize("form", ["resident", "cluster", "colour_phase_plain", "colour_phase_mixed"])
def test_invariants_hold_after_every_window(fk, orc, form):
    cells, nf, nv, nh, seed = (12, 12, 16), (2, 2, 4), 60, 150, 4
    prec = 0 if form == "colour_phase_plain" else 1
    kw = {"resident": dict(schedule=2), "cluster": dict(schedule=2, cluster_ctas=4),
          "colour_phase_plain": dict(schedule=1, small_pass=1),
          "colour_phase_mixed": dict(schedule=1, small_pass=1)}[form]
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], seed, nfrag=nf, precision=prec, cap_v=32, n_tau=2.0, **kw)
    b.set_barriers(0.6, 0.4, 1000.0, field_z=2e7)
    ref = orc.Lattice(cells, nf, nv, nh, seed=seed)
    ref.set_rates(0.6, 0.4, 1000.0, Ez=2e7, a_ang=4.01, cap_v=32, n_tau=2.0, precision=prec)
    check_against_oracle(fk, b, ref, nv, nh)
    for _ in range(12):
        b.run(1)
        ref.run(1)
        check_against_oracle(fk, b, ref, nv, nh)
    assert b.info().hops == ref.counters()["hops"] > 0
    assert b.info().handoffs > 0


def test_invariants_hold_in_the_null_event_form(fk, orc):
    cells, nf, nv, nh, seed = (12, 12, 12), (2, 2, 2), 40, 100, 6
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], seed, nfrag=nf, precision=1, cap_v=32)
    b.set_barriers(0.6, 0.4, 1000.0)
    ref = orc.Lattice(cells, nf, nv, nh, seed=seed)
    ref.set_rates(0.6, 0.4, 1000.0, a_ang=4.01, cap_v=32, precision=1)
    for _ in range(5):
        b.run_null(10, 8)
        ref.null_run(10, 8)
        check_against_oracle(fk, b, ref, nv, nh)


def blob_layout(fk, b, cells):
    """Byte offsets of the occupancy, records and counts in a one-replica blob."""
    n = fk.kmc_state_bytes(b.h)
    rw = (cells[0] + 63) // 64 * 4  # 16 sites per word, rows padded to 16 bytes
    occ_words = 3 * cells[2] * cells[1] * rw
    nfrag = int(np.prod(b.info().nfrag))
    cap = b.info().cap_v
    al = lambda v: (v + 7) & ~7
    o_occ = al(64 + 56)
    o_rec = al(o_occ + 4 * occ_words)
    o_cnt = al(o_rec + 24 * nfrag * cap)
    assert al(o_cnt + 4 * nfrag) == n
    return n, rw, o_occ, o_rec, o_cnt


def test_corrupted_states_are_reported(fk):
    import torch
    cells, nv, nh = (16, 12, 12), 30, 40
    b = fk.Batch([(*cells, 4.01)], [(nv, nh)], 2, edge=4, precision=1, cap_v=32)
    b.set_barriers(0.6, 0.4, 1000.0)
    b.run(10)
    assert b.check().ok == 1
    n, rw, o_occ, o_rec, o_cnt = blob_layout(fk, b, cells)
    good = torch.empty(n, dtype=torch.uint8).pin_memory()
    fk.kmc_download_state(b.h, good.data_ptr(), n)
    g = good.numpy()
    counts = g[o_cnt:o_cnt + 4 * int(np.prod(b.info().nfrag))].view(np.int32)
    f0 = int(np.nonzero(counts > 0)[0][0])  # a fragment holding vacancies, and its first record
    cap = b.info().cap_v
    rec0 = g[o_rec + 24 * f0 * cap:o_rec + 24 * (f0 * cap + 1)]
    key = int(rec0[:8].view(np.uint64)[0])
    x, y, z, t = key & 0xFFFF, (key >> 16) & 0xFFFF, (key >> 32) & 0xFFFF, key >> 48
    word = ((z * cells[1] + y) * rw + (x >> 4)) * 3 + t  # the three site types interleaved per 16-cell block

    def upload_and_check(mutate):
        bad = good.clone().pin_memory()
        mutate(bad.numpy())
        fk.kmc_upload_state(b.h, bad.data_ptr(), n)
        return b.check()

    def clear_vacancy(a):  # V (2) -> O (0) at the record's site
        w = a[o_occ + 4 * word:o_occ + 4 * word + 4].view(np.uint32)
        assert (int(w[0]) >> (2 * (x & 15))) & 3 == fk.FKMC_V
        w[0] &= np.uint32(~(3 << (2 * (x & 15))) & 0xFFFFFFFF)

    inv = upload_and_check(clear_vacancy)
    n_o = 3 * 16 * 12 * 12 - nv - nh + 1
    assert (inv.ok, inv.sites[fk.FKMC_V], inv.sites[fk.FKMC_O], inv.rec_not_vacancy) == (0, nv - 1, n_o, 1)
    assert inv.hash_vac_sites != inv.hash_rec_sites

    def change_id(a):
        a[o_rec + 24 * f0 * cap + 20:o_rec + 24 * f0 * cap + 24].view(np.uint32)[0] += np.uint32(nv)

    inv = upload_and_check(change_id)
    assert (inv.ok, inv.rec_not_vacancy) == (0, 0) and inv.hash_rec_ids != inv.hash_ids_expected

    def count_over_cap(a):
        a[o_cnt + 4 * f0:o_cnt + 4 * f0 + 4].view(np.int32)[0] = cap + 1

    inv = upload_and_check(count_over_cap)
    assert (inv.ok, inv.frag_bad_count) == (0, 1)

    fk.kmc_upload_state(b.h, good.data_ptr(), n)  # back to the consistent state, which runs on
    assert b.check().ok == 1
    b.run(5)
    assert b.check().ok == 1

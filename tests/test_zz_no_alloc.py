"""kmc_vacancy_moments_noalloc: the allocation-free moment reduction, for
callers that cannot allocate device memory (a framework that owns every device
allocation, a plugin handed fixed buffers).  Its output must equal the
batch's own kmc_read_moments_all on the same records, on two calls in a row
(the static scratch keeps the previous call's contents and must be cleared).
Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REC = np.dtype([("key", "<u8"), ("d", "<i4", (3,)), ("id", "<u4")])


def test_noalloc_moments_match_batch_reduction():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_09081_gb300 import fkmc
    fkmc.load()
    cells = [(8, 8, 8), (12, 10, 8), (16, 16, 16), (9, 9, 9), (6, 8, 10)]
    comps = [(15, 0), (20, 40), (60, 300), (3, 10), (12, 30)]
    b = fkmc.Batch([(*c, 4.01) for c in cells], comps, 5, edge=4, precision=1, cap_v=32)
    b.set_barriers(0.7, 0.35, [800.0, 650.0, 900.0, 1000.0, 700.0])
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        b.run(30)
        ref = b.moments_all()
        # the same records, copied into buffers this test owns
        cap = b.info(0).cap_v
        nfr = [int(np.prod(list(b.info(r).nfrag))) for r in range(b.n)]
        offsets = np.concatenate([[0], np.cumsum(nfr)]).astype(np.int64)
        recs = np.zeros(offsets[-1] * cap, REC)
        counts = np.zeros(offsets[-1], np.int32)
        for r in range(b.n):
            for f, site, dx, dy, dz, vid in b.records(r):
                g = offsets[r] + f
                k = g * cap + counts[g]
                recs[k]["key"] = site
                recs[k]["d"] = (dx, dy, dz)
                recs[k]["id"] = vid
                counts[g] += 1
        d_recs = torch.from_numpy(recs.view(np.uint8)).cuda()
        d_counts = torch.from_numpy(counts).cuda()
        torch.cuda.synchronize()
        got = fkmc.kmc_vacancy_moments_noalloc(d_recs.data_ptr(), d_counts.data_ptr(), offsets, cap, stream)
        assert np.array_equal(got, ref), (call, got, ref)
        assert got[:, 0].tolist() == [c[0] for c in comps]
    # sizes beyond the static scratch are rejected, not truncated
    too_many = np.zeros(fkmc.FKMC_NOALLOC_MAX_GROUPS + 2, np.int64)
    with pytest.raises(fkmc.KmcError) as e:
        fkmc.kmc_vacancy_moments_noalloc(d_recs.data_ptr(), d_counts.data_ptr(), too_many, cap, stream)
    assert e.value.code == fkmc.FKMC_EINVAL


def _numpy_moments(recs, counts, offsets, cap):
    out = np.zeros((len(offsets) - 1, 7), np.int64)
    for g in range(len(offsets) - 1):
        for f in range(offsets[g], offsets[g + 1]):
            d = recs[f * cap: f * cap + counts[f]]["d"].astype(np.int64)
            out[g, 0] += len(d)
            out[g, 1:4] += d.sum(0)
            out[g, 4:7] += (d * d).sum(0)
    return out


@pytest.mark.parametrize("n_groups,empty_every", [(4096, 3), (37, 2)])
def test_noalloc_at_the_group_limit_and_with_empty_groups(n_groups, empty_every):
    """At FKMC_NOALLOC_MAX_GROUPS groups (the last offset and accumulator of
    the static scratch in use) and with empty groups between non-empty ones
    (equal offsets: the group search must give each record to the group that
    owns its fragment), on two calls in a row, against numpy sums."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_09081_gb300 import fkmc
    fkmc.load()
    rng = np.random.default_rng(n_groups)
    cap = 8
    sizes = rng.integers(1, 4, n_groups)
    sizes[::empty_every] = 0          # empty groups, including the first
    sizes[-1] = max(sizes[-1], 1)     # the last group holds records
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    nfrag = int(offsets[-1])
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        counts = rng.integers(0, cap + 1, nfrag).astype(np.int32)
        recs = np.zeros(nfrag * cap, REC)
        recs["d"] = rng.integers(-50, 51, (nfrag * cap, 3))
        recs["key"] = rng.integers(0, 2**40, nfrag * cap)
        d_recs = torch.from_numpy(recs.view(np.uint8)).cuda()
        d_counts = torch.from_numpy(counts).cuda()
        torch.cuda.synchronize()
        got = fkmc.kmc_vacancy_moments_noalloc(d_recs.data_ptr(), d_counts.data_ptr(), offsets, cap, stream)
        assert np.array_equal(got, _numpy_moments(recs, counts, offsets, cap)), call
        assert (got[sizes == 0] == 0).all()

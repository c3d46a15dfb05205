"""Pins of the oracle's primitives against things other than itself.

- Philox4x64-10 against numpy's independent Philox bit generator.
- The two series logarithms against libm (math.log).
- The neighbour table against a real-space distance search done here.
- The placement bijection, colour permutation and partition by their
  defining properties.
- The rate table against its closed form and the detailed-balance ratio.
"""
import math

import numpy as np
import pytest

M64 = (1 << 64) - 1


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(1)
    for _ in range(300):
        c = [int(v) for v in rng.integers(0, 2**63, 4, dtype=np.uint64)]
        k = [int(v) for v in rng.integers(0, 2**64 - 1, 2, dtype=np.uint64)]
        # numpy's Philox returns the block of counter+1 first
        bg = np.random.Philox(counter=np.array(c, np.uint64), key=np.array(k, np.uint64))
        ref = bg.random_raw(4)
        c1 = list(c)
        c1[0] = (c1[0] + 1) & M64
        got = orc.philox4x64(c1, k)
        assert np.array_equal(got, ref)


def test_philox_small_counters(orc):
    for c, k in [([0, 0, 0, 0], [0, 0]), ([0, 7, 0, 0], [3, 0]), ([9, 0, 2, 1], [0, 13])]:
        bg = np.random.Philox(counter=np.array(c, np.uint64), key=np.array(k, np.uint64))
        ref = bg.random_raw(4)
        c1 = list(c)
        c1[0] += 1
        assert np.array_equal(orc.philox4x64(c1, k), ref)


def _u53(x):
    return (2 * (x >> 12) + 1) * 2.0**-53


def test_neglog64_against_libm(orc):
    """Within 1 ulp of libm's log on 1e7 points (uniform words, and words
    shifted right by a random amount so that every binary exponent of u is
    covered), and correctly rounded on the large majority of them."""
    rng = np.random.default_rng(2)
    n = 10_000_000
    x = rng.integers(0, 2**64 - 1, n, dtype=np.uint64, endpoint=True)
    sh = rng.integers(0, 64, n // 4, dtype=np.uint64)
    x[1::4] = x[1::4] >> sh
    edge = np.array([0, 1, 4095, 4096, 2**63, M64, M64 - 4096, 2**52, 3 << 60], np.uint64)
    x = np.concatenate([x, edge])
    u = (2 * (x >> np.uint64(12)) + np.uint64(1)).astype(np.float64) * 2.0**-53  # exact
    got = orc.neglog64_batch(x)
    ref = np.array([-math.log(v) for v in u.tolist()])
    ulps = np.abs(got.view(np.int64) - ref.view(np.int64))
    assert ulps.max() <= 1, int(ulps.max())
    assert (ulps == 0).mean() > 0.9


def test_neglog64_extremes(orc):
    assert orc.neglog64(0) == pytest.approx(53 * math.log(2), rel=1e-15)
    assert orc.neglog64(M64) == pytest.approx(2.0**-53, rel=1e-6)


def _u32(x):
    """u of the FP32 form: leading one, next 22 bits, forced midpoint bit."""
    x |= 1
    p = x.bit_length() - 1
    nx = (x << (63 - p)) & M64
    mant = (nx >> 40) | 1
    return mant * 2.0**-23 * 2.0 ** (p - 64)


def test_neglog32_against_libm(orc):
    rng = np.random.default_rng(3)
    xs = [int(v) for v in rng.integers(0, 2**64 - 1, 20000, dtype=np.uint64)]
    xs += [0, 1, 2, 3, 2**63, M64, 1 << 40, (1 << 41) - 1]
    for x in xs:
        u = _u32(x)
        ref = -math.log(u)
        got = orc.neglog32(x)
        # fp32 arithmetic: a few float ulps of the larger of the two terms
        assert abs(got - ref) <= 4 * 2.0**-23 * max(1.0, ref), (x, got, ref)
        # and the draw is within 2^-23 (relative) of the exact uniform x/2^64
        assert abs(u - (x | 1) / 2.0**64) <= 2.0**-22 * u


def test_neglog_distribution_is_exponential(orc):
    """Mean and second moment of -ln u over Philox draws: Exp(1) has 1 and 2."""
    k = [5, 0]
    e64, e32 = [], []
    for i in range(20000):
        y = orc.philox4x64([i, 0, 0, 0], k)
        e64.append(orc.neglog64(int(y[0])))
        e32.append(orc.neglog32(int(y[1])))
    for e in (np.array(e64), np.array(e32)):
        assert abs(e.mean() - 1.0) < 4 / math.sqrt(len(e))
        assert abs((e**2).mean() - 2.0) < 4 * math.sqrt(20) / math.sqrt(len(e))


def test_neighbour_table_real_space(orc):
    """Every O site has exactly 8 nearest O neighbours at a/sqrt2; the table
    lists them in ascending (dx,dy,dz) and the relation is symmetric."""
    tab = orc.neighbour_table()
    e = np.eye(3, dtype=int)
    # positions in units of a/2 of all sites in a 5^3 block around cell 0
    sites = []
    for t in range(3):
        for c in np.ndindex(5, 5, 5):
            c = np.array(c) - 2
            sites.append((t, tuple(c), 2 * c + e[t]))
    for t in range(3):
        p0 = e[t]
        near = []
        for (t2, c, p) in sites:
            d = p - p0
            r2 = int(d @ d)
            if r2 == 0:
                continue
            near.append((r2, tuple(d), t2, c))
        rmin = min(n[0] for n in near)
        assert rmin == 2  # (a/2)^2 * 2 = a^2/2 -> distance a/sqrt2
        first = sorted((n for n in near if n[0] == rmin), key=lambda n: n[1])
        assert len(first) == 8
        for n, (r2, d, t2, c) in enumerate(first):
            row = tab[t, n]
            assert row[0] == t2
            assert tuple(row[1:4]) == c
            assert tuple(row[4:7]) == d
    # symmetry: the reverse hop exists in the neighbour's table
    for t in range(3):
        for n in range(8):
            t2, d = tab[t, n, 0], tuple(-tab[t, n, 4:7])
            assert any(tuple(tab[t2, m, 4:7]) == d and tab[t2, m, 0] == t for m in range(8))


@pytest.mark.parametrize("nsite", [1, 2, 3, 24, 1000, 1536, 98304])
def test_feistel_is_a_permutation(orc, nsite):
    k = min(nsite, 2000)
    vals = [orc.feistel(i, nsite, 7) for i in range(k)]
    assert len(set(vals)) == k
    assert all(0 <= v < nsite for v in vals)
    if nsite <= 2000:
        assert sorted(vals) == list(range(nsite))


def test_feistel_placement_is_uniform(orc):
    nsite = 24
    counts = np.zeros(nsite)
    for seed in range(3000):
        counts[orc.feistel(0, nsite, seed)] += 1
    exp = 3000 / nsite
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 60  # df = 23; p ~ 3e-5


def test_colour_permutation(orc):
    firsts = np.zeros(8)
    for w in range(4000):
        p = orc.colour_perm(11, 3, w)
        assert sorted(p) == list(range(8))
        firsts[p[0]] += 1
    exp = 500
    assert ((firsts - exp) ** 2 / exp).sum() < 30  # df = 7


def test_rate_table_closed_form(orc):
    kB = 8.617333262e-5
    T, Ea_O, Ea_H, A, a = 800.0, 0.6, 0.3, 1e13, 3.905
    k64, k32, q, F = orc.rate_table(Ea_O, Ea_H, A, 2.0, 1.0, T, 0.0, a)
    assert k64[:3] == pytest.approx([A * math.exp(-Ea_O / (kB * T))] * 3, rel=1e-14)
    assert k64[3:] == pytest.approx([A * math.exp(-Ea_H / (kB * T))] * 3, rel=1e-14)
    assert F == 63 - 9  # C_v = 64 -> 8*64 = 2^9 events
    assert np.all(k32 == k64.astype(np.float32))
    assert q.max() == 2**F
    # fixed point keeps the fp32 ratio to 2^-F
    assert q[0] / 2.0**F == pytest.approx(float(k32[0]) / float(k32.max()), abs=2.0**-F)


def test_rate_table_field_detailed_balance(orc):
    """Under a uniform field along z, forward/backward rates differ by
    exp(-dU/kT) (detailed balance) and in-plane hops are unchanged."""
    kB = 8.617333262e-5
    T, Ez, a = 400.0, 1e7, 4.01
    k64, _, _, _ = orc.rate_table(0.7, 0.35, 1e13, 2.0, 1.0, T, Ez, a)
    for h, qc in ((0, 2.0), (1, 1.0)):
        down, flat, up = k64[3 * h], k64[3 * h + 1], k64[3 * h + 2]
        dU_up = -qc * Ez * 0.5 * a * 1e-10  # vacancy moves +a/2 along the field
        assert up / down == pytest.approx(math.exp(-dU_up / (kB * T)), rel=1e-12)
        assert flat == pytest.approx(up * down / flat, rel=1e-12)  # geometric mean
    assert k64[2] > k64[0]  # the vacancy (positive) drifts along +z


def test_partition_rejects_bad_fragmentations(orc):
    with pytest.raises(ValueError):
        orc.Lattice((8, 8, 8), (3, 2, 2), 1, 0)  # odd count
    with pytest.raises(ValueError):
        orc.Lattice((6, 8, 8), (4, 2, 2), 1, 0)  # edge < 2
    orc.Lattice((8, 8, 8), (1, 2, 4), 1, 0)


def test_initial_state_counts(orc):
    L = orc.Lattice((8, 8, 8), (2, 2, 2), 15, 40, seed=3)
    occ = L.occupancy()
    assert np.bincount(occ, minlength=3).tolist() == [1536 - 55, 40, 15]
    rec = L.records()
    assert len(rec) == 15
    assert sorted(rec[:, 5].tolist()) == list(range(15))
    assert set(rec[:, 1].tolist()) == set(np.flatnonzero(occ == 2).tolist())


def test_partition_reading(orc):
    """Fragments per dimension for a target edge: the even count nearest L/e
    with every edge floor(L/n) or ceil(L/n) >= 2 cells.  Pinned to the
    partitions the workloads are specified with (8^3 cells in 2^3 fragments of
    4^3, 32^3 in 8^3 of 4^3, 128^3 in 16^3 of 8^3, 2500 cells of edge-8
    fragments: 312 fragments, 308 of 8 cells and 4 of 9) and to its defining
    properties on every L <= 160, e <= 12."""
    assert orc.partition((8, 8, 8), 4) == (2, 2, 2)
    assert orc.partition((32, 32, 32), 4) == (8, 8, 8)
    assert orc.partition((128, 128, 128), 8) == (16, 16, 16)
    n = orc.partition((2500,), 8)[0]
    base, rem = divmod(2500, n)
    assert (n, base, rem, n - rem) == (312, 8, 4, 308)
    for L in range(1, 161):
        for e in range(1, 13):
            n = orc.partition((L,), e)[0]
            if L < 4:
                assert n == 1
                continue
            assert n % 2 == 0 and L // n >= 2
            # the even count nearest L/e (2 round(L/2e), half up), clamped to the valid range
            want = 2 * math.floor(L / (2 * e) + 0.5)
            want = min(max(want, 2), 2 * (L // 4))
            assert n == want, (L, e, n, want)

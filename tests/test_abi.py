"""The C-ABI library loads and exports every entry point of include/*.h;
its host-only helpers agree with the oracle bit for bit (no GPU needed)."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_09081_gb300 import _build, fkmc
    _build.build()
    return fkmc


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(kmc_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_abi():
    names = declared_functions()
    for must in ("kmc_create_lattice", "kmc_set_barriers", "kmc_run", "kmc_read_msd", "kmc_read_D",
                 "kmc_create_batch", "kmc_destroy", "kmc_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.load()
    for name in declared_functions():
        assert hasattr(L, name), name
    # the binding wraps every entry point under the same name
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_defaults(lib):
    o = lib.kmc_default_opts()
    assert o.edge == 4 and o.precision == 0 and o.n_tau == 1.0 and o.cap_v == 0 and o.cluster_top == -1


def test_neighbour_table_matches_oracle(lib, orc):
    assert np.array_equal(lib.kmc_neighbour_table(), orc.neighbour_table())


@pytest.mark.parametrize("T,Ez,a,cap", [(800.0, 0.0, 3.905, 64), (400.0, 1e7, 4.01, 32),
                                        (300.0, -3e8, 4.01, 256), (1000.0, 5e6, 3.905, 8)])
def test_rate_table_bits_match_oracle(lib, orc, T, Ez, a, cap):
    tab = lib.kmc_barrier_table(0.7, 0.35, 1e13, 2.0, 1.0)
    k64, k32, q, F = lib.kmc_rate_table(tab, T, Ez, a, cap)
    r64, r32, rq, rF = orc.rate_table(0.7, 0.35, 1e13, 2.0, 1.0, T, Ez, a, cap)
    assert F == rF
    assert np.array_equal(k64.view(np.uint64), r64.view(np.uint64))
    assert np.array_equal(k32.view(np.uint32), r32.view(np.uint32))
    assert np.array_equal(q, rq)


def test_rate_table_rejects_bad_input(lib):
    tab = lib.kmc_barrier_table(0.7, 0.35, 1e13, 2.0, 1.0)
    with pytest.raises(lib.KmcError) as e:
        lib.kmc_rate_table(tab, -1.0, 0.0, 4.0, 64)
    assert e.value.code == lib.FKMC_EINVAL


def test_site_shell_tables_match_oracle(lib):
    """The library's interaction partners (built from displacement vectors)
    equal the oracle's (built from a cell search), energies included."""
    import oracle as orc
    vv = [(2, 0.343), (4, 0.235), (6, 0.200), (8, 0.180), (10, 0.023), (16, 0.011)]
    fe = [(1, -0.709), (5, -0.199), (9, -0.022), (13, 0.0005)]
    ref = orc.Lattice((9, 9, 9), (1, 1, 1), 0, 0)
    ref.set_site_energy(vv=vv, fe=fe)
    for t in range(3):
        got = sorted(map(tuple, lib.kmc_site_shells(vv, fe, t).tolist()))
        want = sorted(map(tuple, ref.shells(t).tolist()))
        assert got == want
    with pytest.raises(lib.KmcError):
        lib.kmc_site_shells([(3, 0.1)], [], 0)  # not an O-O distance
    with pytest.raises(lib.KmcError):
        lib.kmc_site_shells([(2, 0.1), (2, 0.2)], [], 0)  # listed twice


@pytest.mark.parametrize("field,value", [("small_pass", 3), ("small_pass", -2), ("schedule", 3), ("precision", 5),
                                         ("cap_v", 12), ("n_tau", 0.0), ("n_tau", 65.0), ("lane_form", 3),
                                         ("lane_form", -1), ("cluster_ctas", 1), ("cluster_ctas", -2),
                                         ("cluster_ctas", 17)])
def test_create_batch_rejects_bad_options(lib, field, value):
    """Options are checked before any device work: a bad value is FKMC_EINVAL
    (so this runs without a GPU)."""
    o = lib.kmc_default_opts()
    setattr(o, field, value)
    with pytest.raises(lib.KmcError) as e:
        lib.kmc_create_batch([lib.kmc_cells(8, 8, 8, 3.905)], [lib.kmc_composition(5, 0, 0)], 0, o)
    assert e.value.code == lib.FKMC_EINVAL


def test_default_options_of_the_run_passes(lib):
    o = lib.kmc_default_opts()
    assert o.small_pass == 0 and o.schedule == 0 and o.cluster_top == -1 and o.lane_form == 0
    assert o.cluster_ctas == 0


@pytest.mark.parametrize("tracer,n_fe", [(0, 0), (1, 0), (0, 3)])
def test_allocation_failure_is_enomem_and_frees_everything(lib, tracer, n_fe):
    """Failure injected on the host: the caller's allocator returns NULL from
    its k-th call on, for every k.  kmc_create_batch must return FKMC_ENOMEM
    and hand every block it did get back to the caller's free.  The allocator
    never returns a full set of blocks, so the library never touches one on
    the device: this runs with or without a GPU."""
    import ctypes as C

    def attempt(k):
        got, freed = [], []

        def alloc(ctx, n):
            if len(got) + 1 >= k:
                got.append(None)
                return None
            got.append(0x10000 * (len(got) + 1))  # distinct, never dereferenced
            return got[-1]

        def free(ctx, p):
            freed.append(p)

        ca, cf = lib.kmc_alloc_fn(alloc), lib.kmc_free_fn(free)
        o = lib.kmc_default_opts()
        o.tracer = tracer
        o.cluster_top = 0
        o.alloc, o.free = ca, cf
        with pytest.raises(lib.KmcError) as e:
            lib.kmc_create_batch([lib.kmc_cells(8, 8, 8, 3.905), lib.kmc_cells(6, 6, 6, 3.905)],
                                 [lib.kmc_composition(5, 3, n_fe), lib.kmc_composition(2, 0, n_fe)], 0, o)
        assert e.value.code == lib.FKMC_ENOMEM
        assert sorted(freed) == sorted(p for p in got if p is not None)
        return len(got)

    total = attempt(1)  # every call fails: counts the allocations of a batch
    assert total >= 14
    for k in range(2, total + 1):
        attempt(k)


def test_create_batch_rejects_bad_wait_test_option(lib):
    o = lib.kmc_default_opts()
    o.test_stuck_wait_us = -1
    with pytest.raises(lib.KmcError) as e:
        lib.kmc_create_batch([lib.kmc_cells(8, 8, 8, 3.905)], [lib.kmc_composition(5, 0, 0)], 0, o)
    assert e.value.code == lib.FKMC_EINVAL


def test_partition_matches_the_oracles_reading(lib, orc):
    """The library's fragment count per dimension (a closed form) equals the
    oracle's (a search over even counts) on every L <= 300 and edge 1..12."""
    for L in range(1, 301):
        for e in range(1, 13):
            assert lib.kmc_partition_count(L, e) == orc.partition((L,), e)[0], (L, e)
    assert lib.kmc_partition_count(0, 4) == 0 and lib.kmc_partition_count(8, 0) == 0

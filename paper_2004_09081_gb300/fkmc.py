"""Thin ctypes binding of the C ABI in include/fkmc.h.

Every function named ``kmc_*`` here has the C entry point's name and does
argument marshalling only; all work happens in the CUDA library.  Device
memory comes from PyTorch's caching allocator through the ABI's allocator
callback, and work goes to the current torch CUDA stream.  If the compiled
library is missing, importing the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

FKMC_OK, FKMC_EINVAL, FKMC_ENOMEM, FKMC_ECUDA, FKMC_ETIMEOUT, FKMC_EOVERFLOW, FKMC_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
FKMC_O, FKMC_H, FKMC_V = 0, 1, 2
FKMC_PLAIN, FKMC_MIXED = 0, 1


class KmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fkmc error {code}: {msg}")
        self.code = code


class kmc_cells(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("a_angstrom", C.c_double)]


class kmc_composition(C.Structure):
    _fields_ = [("n_vac", C.c_int64), ("n_H", C.c_int64), ("n_Fe", C.c_int64)]


FKMC_MAX_SHELLS = 8


class kmc_site_energy(C.Structure):
    _fields_ = [("n_vv", C.c_int32), ("vv_d2", C.c_int32 * FKMC_MAX_SHELLS), ("vv_eV", C.c_double * FKMC_MAX_SHELLS),
                ("n_fe", C.c_int32), ("fe_d2", C.c_int32 * FKMC_MAX_SHELLS), ("fe_eV", C.c_double * FKMC_MAX_SHELLS)]


class kmc_grains(C.Structure):
    _fields_ = [("n_grains", C.c_int32), ("width", C.c_int32), ("barrier_eV", C.c_double)]


class kmc_electrostatics(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("q_vac", C.c_double), ("refresh_windows", C.c_int32),
                ("cycles", C.c_int32), ("warm_cycles", C.c_int32)]


class kmc_barrier_table(C.Structure):
    _fields_ = [("Ea_O_eV", C.c_double), ("Ea_H_eV", C.c_double), ("prefactor", C.c_double),
                ("q_O", C.c_double), ("q_H", C.c_double)]


kmc_alloc_fn = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
kmc_free_fn = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class kmc_opts(C.Structure):
    _fields_ = [("edge", C.c_int32), ("nfrag", C.c_int32 * 3), ("precision", C.c_int32),
                ("tracer", C.c_int32), ("cap_v", C.c_int32), ("n_tau", C.c_double),
                ("stream", C.c_void_p), ("alloc", kmc_alloc_fn), ("free", kmc_free_fn),
                ("alloc_ctx", C.c_void_p), ("schedule", C.c_int32), ("cluster_top", C.c_int32),
                ("small_pass", C.c_int32), ("test_stuck_wait_us", C.c_int32), ("lane_form", C.c_int32),
                ("cluster_ctas", C.c_int32), ("reserved", C.c_int32 * 2)]


class kmc_run_stats(C.Structure):
    _fields_ = [("hops", C.c_uint64), ("handoffs", C.c_uint64), ("windows", C.c_uint64),
                ("gpu_ms", C.c_double), ("launches", C.c_uint64)]


class kmc_replica_info(C.Structure):
    _fields_ = [("nfrag", C.c_int32 * 3), ("cap_v", C.c_int32), ("F", C.c_int32),
                ("precision", C.c_int32), ("tau", C.c_double), ("theta_tau", C.c_double),
                ("k64", C.c_double * 6), ("q", C.c_uint64 * 6), ("window", C.c_uint64),
                ("hops", C.c_uint64), ("handoffs", C.c_uint64), ("nsite", C.c_int64),
                ("n_vac", C.c_int64), ("n_H", C.c_int64), ("null_steps", C.c_uint64),
                ("null_theta", C.c_double), ("null_time_s", C.c_double), ("n_Fe", C.c_int64),
                ("kernel", C.c_int32), ("ctas", C.c_int32), ("draw_phases", C.c_int32), ("draw_events", C.c_int32)]


class kmc_invariants(C.Structure):
    _fields_ = [("sites", C.c_int64 * 4), ("records", C.c_int64), ("rec_not_vacancy", C.c_int64),
                ("rec_wrong_fragment", C.c_int64), ("rec_outside", C.c_int64), ("frag_bad_count", C.c_int64),
                ("hash_vac_sites", C.c_uint64), ("hash_rec_sites", C.c_uint64), ("hash_rec_ids", C.c_uint64),
                ("hash_ids_expected", C.c_uint64), ("ok", C.c_int32), ("pad", C.c_int32)]


_P, _I32, _I64, _U64, _SZ, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_size_t, C.c_double
_SIGNATURES = {
    "kmc_default_opts": (None, [_P]),
    "kmc_create_batch": (C.c_int, [_I32, _P, _P, _U64, _P, _P]),
    "kmc_create_lattice": (C.c_int, [_P, _P, _U64, _P, _P]),
    "kmc_set_barriers": (C.c_int, [_P, _P, _P, _P]),
    "kmc_run": (C.c_int, [_P, _U64, _P]),
    "kmc_run_null": (C.c_int, [_P, _U64, _I64, _P]),
    "kmc_read_moments": (C.c_int, [_P, _I32, _I32, _P]),
    "kmc_read_moments_all": (C.c_int, [_P, _P, _SZ]),
    "kmc_read_msd": (C.c_int, [_P, _I32, _I32, _P, _P, _P]),
    "kmc_read_D": (C.c_int, [_P, _I32, _I32, _P, _P, _P, _P]),
    "kmc_read_state": (C.c_int, [_P, _I32, _P, _SZ]),
    "kmc_write_state": (C.c_int, [_P, _I32, _P, _SZ]),
    "kmc_read_records": (C.c_int, [_P, _I32, _P, _I64, _P]),
    "kmc_read_tracer": (C.c_int, [_P, _I32, _P, _SZ]),
    "kmc_state_bytes": (C.c_int, [_P, _P]),
    "kmc_download_state": (C.c_int, [_P, _P, _SZ]),
    "kmc_upload_state": (C.c_int, [_P, _P, _SZ]),
    "kmc_get_replica_info": (C.c_int, [_P, _I32, _P]),
    "kmc_check_invariants": (C.c_int, [_P, _I32, _P]),
    "kmc_num_replicas": (_I32, [_P]),
    "kmc_rate_table": (C.c_int, [_P, _D, _D, _D, _I32, _P, _P, _P, _P]),
    "kmc_neighbour_table": (None, [_P]),
    "kmc_partition_count": (_I32, [_I32, _I32]),
    "kmc_vacancy_moments_noalloc": (C.c_int, [_P, _P, _P, _I32, _I32, _P, _P]),
    "kmc_set_site_energy": (C.c_int, [_P, _P]),
    "kmc_read_dopants": (C.c_int, [_P, _I32, _P, _SZ]),
    "kmc_write_dopants": (C.c_int, [_P, _I32, _P, _SZ]),
    "kmc_read_site_field": (C.c_int, [_P, _I32, _P, _SZ]),
    "kmc_site_shells": (C.c_int, [_P, _I32, _P, _I32, _P]),
    "kmc_set_grains": (C.c_int, [_P, _P]),
    "kmc_set_electrostatics": (C.c_int, [_P, _P]),
    "kmc_solve_potential": (C.c_int, [_P, _I32, _P, _SZ, _P]),
    "kmc_read_potential_energy": (C.c_int, [_P, _I32, _P, _SZ, _P]),
    "kmc_write_potential_energy": (C.c_int, [_P, _I32, _P, _SZ, _P]),
    "kmc_read_grains": (C.c_int, [_P, _I32, _P, _P, _SZ]),
    "kmc_destroy": (C.c_int, [_P]),
    "kmc_last_error": (C.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load the compiled library (never builds implicitly; see __graft_entry__.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"fkmc CUDA library not built: {_build.LIB} is missing "
                              "(run __graft_entry__.build())")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != FKMC_OK:
        raise KmcError(rc, load().kmc_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------ ABI functions
def kmc_default_opts() -> kmc_opts:
    o = kmc_opts()
    load().kmc_default_opts(C.byref(o))
    return o


def kmc_create_batch(cells, comps, seed: int, opts: kmc_opts) -> C.c_void_p:
    n = len(cells)
    ca = (kmc_cells * n)(*cells)
    co = (kmc_composition * n)(*comps)
    h = C.c_void_p()
    _check(load().kmc_create_batch(n, ca, co, int(seed), C.byref(opts), C.byref(h)))
    return h


def kmc_create_lattice(cells: kmc_cells, comp: kmc_composition, seed: int, opts: kmc_opts):
    h = C.c_void_p()
    _check(load().kmc_create_lattice(C.byref(cells), C.byref(comp), int(seed), C.byref(opts), C.byref(h)))
    return h


def kmc_set_barriers(h, tables, T_K, field_z):
    n = len(tables)
    ta = (kmc_barrier_table * n)(*tables)
    T = np.ascontiguousarray(T_K, np.float64)
    E = np.ascontiguousarray(field_z, np.float64)
    _check(load().kmc_set_barriers(h, ta, _ptr(T), _ptr(E)))


def kmc_run(h, windows: int) -> kmc_run_stats:
    s = kmc_run_stats()
    _check(load().kmc_run(h, int(windows), C.byref(s)))
    return s


def kmc_run_null(h, steps: int, n_frg: int) -> kmc_run_stats:
    s = kmc_run_stats()
    _check(load().kmc_run_null(h, int(steps), int(n_frg), C.byref(s)))
    return s


def kmc_read_moments(h, r: int, species: int) -> np.ndarray:
    out = np.zeros(7, np.int64)
    _check(load().kmc_read_moments(h, r, species, _ptr(out)))
    return out


def kmc_read_moments_all(h, n: int) -> np.ndarray:
    out = np.zeros((n, 7), np.int64)
    _check(load().kmc_read_moments_all(h, _ptr(out), out.size))
    return out


def kmc_read_msd(h, r: int, species: int):
    msd, mean, t = np.zeros(3), np.zeros(3), C.c_double()
    _check(load().kmc_read_msd(h, r, species, _ptr(msd), _ptr(mean), C.byref(t)))
    return msd, mean, t.value


def kmc_read_D(h, r: int, species: int):
    """(D_xyz drift-removed per axis, D = MSD/6t, D_xy, v_drift[3]); m^2/s, m/s."""
    Dx, D, Dxy, v = np.zeros(3), C.c_double(), C.c_double(), np.zeros(3)
    _check(load().kmc_read_D(h, r, species, _ptr(Dx), C.byref(D), C.byref(Dxy), _ptr(v)))
    return Dx, D.value, Dxy.value, v


def kmc_read_state(h, r: int, nsite: int) -> np.ndarray:
    out = np.zeros(nsite, np.uint8)
    _check(load().kmc_read_state(h, r, _ptr(out), nsite))
    return out


def kmc_write_state(h, r: int, occ: np.ndarray):
    occ = np.ascontiguousarray(occ, np.uint8)
    _check(load().kmc_write_state(h, r, _ptr(occ), occ.size))


def kmc_read_records(h, r: int) -> np.ndarray:
    n = C.c_int64()
    _check(load().kmc_read_records(h, r, None, 0, C.byref(n)))
    out = np.zeros((max(n.value, 1), 6), np.int64)
    _check(load().kmc_read_records(h, r, _ptr(out), n.value, C.byref(n)))
    return out[: n.value]


def kmc_read_tracer(h, r: int, nsite: int) -> np.ndarray:
    out = np.zeros((nsite, 3), np.int32)
    _check(load().kmc_read_tracer(h, r, _ptr(out), nsite))
    return out


def kmc_state_bytes(h) -> int:
    n = C.c_size_t()
    _check(load().kmc_state_bytes(h, C.byref(n)))
    return n.value


def kmc_download_state(h, host_ptr: int, nbytes: int):
    _check(load().kmc_download_state(h, C.c_void_p(host_ptr), nbytes))


def kmc_upload_state(h, host_ptr: int, nbytes: int):
    _check(load().kmc_upload_state(h, C.c_void_p(host_ptr), nbytes))


def kmc_get_replica_info(h, r: int) -> kmc_replica_info:
    info = kmc_replica_info()
    _check(load().kmc_get_replica_info(h, r, C.byref(info)))
    return info


def kmc_check_invariants(h, r: int) -> kmc_invariants:
    inv = kmc_invariants()
    _check(load().kmc_check_invariants(h, r, C.byref(inv)))
    return inv


def kmc_num_replicas(h) -> int:
    return int(load().kmc_num_replicas(h))


def kmc_rate_table(table: kmc_barrier_table, T_K: float, field_z: float, a_ang: float, cap_v: int):
    k64, k32, q = np.zeros(6), np.zeros(6, np.float32), np.zeros(6, np.uint64)
    F = C.c_int32()
    _check(load().kmc_rate_table(C.byref(table), T_K, field_z, a_ang, cap_v, _ptr(k64), _ptr(k32),
                                 _ptr(q), C.byref(F)))
    return k64, k32, q, F.value


def kmc_partition_count(L: int, edge: int) -> int:
    return int(load().kmc_partition_count(int(L), int(edge)))


def kmc_neighbour_table() -> np.ndarray:
    out = np.zeros((3, 8, 7), np.int32)
    load().kmc_neighbour_table(_ptr(out))
    return out


FKMC_NOALLOC_MAX_GROUPS = 4096


def kmc_vacancy_moments_noalloc(records_ptr: int, counts_ptr: int, fragment_offsets, cap_v: int,
                                stream_ptr: int = 0) -> np.ndarray:
    """Moments per group from caller-owned device buffers; the library
    allocates nothing for this call (scratch is a static device array)."""
    off = np.ascontiguousarray(fragment_offsets, np.int64)
    n = off.size - 1
    out = np.zeros((max(n, 1), 7), np.int64)
    _check(load().kmc_vacancy_moments_noalloc(C.c_void_p(records_ptr), C.c_void_p(counts_ptr), _ptr(off), n,
                                               int(cap_v), _ptr(out), C.c_void_p(stream_ptr)))
    return out[:n]


def kmc_set_site_energy(h, vv=(), fe=()):
    """vv, fe: sequences of (squared distance in (a/2)^2, energy in eV); both
    empty turns the interactions off."""
    if not vv and not fe:
        _check(load().kmc_set_site_energy(h, None))
        return
    e = _site_energy_struct(vv, fe)
    _check(load().kmc_set_site_energy(h, C.byref(e)))


def _site_energy_struct(vv, fe) -> kmc_site_energy:
    e = kmc_site_energy()
    e.n_vv = len(vv)
    e.n_fe = len(fe)
    for k, (d2, en) in enumerate(vv):
        e.vv_d2[k] = int(d2)
        e.vv_eV[k] = float(en)
    for k, (d2, en) in enumerate(fe):
        e.fe_d2[k] = int(d2)
        e.fe_eV[k] = float(en)
    return e


def kmc_site_shells(vv, fe, t: int) -> np.ndarray:
    e = _site_energy_struct(vv, fe)
    n = C.c_int32()
    _check(load().kmc_site_shells(C.byref(e), int(t), None, 0, C.byref(n)))
    out = np.zeros((max(n.value, 1), 5), np.int32)
    _check(load().kmc_site_shells(C.byref(e), int(t), _ptr(out), n.value, C.byref(n)))
    return out[: n.value]


def kmc_set_electrostatics(h, eps_r=None, q_vac=2.0, refresh_windows=8, cycles=12, warm_cycles=0):
    """Potential of the vacancy charges (multigrid), refreshed every
    refresh_windows windows (warm_cycles V-cycles from the last potential, 0:
    cycles); eps_r None turns it off."""
    if eps_r is None:
        _check(load().kmc_set_electrostatics(h, None))
        return
    e = kmc_electrostatics(float(eps_r), float(q_vac), int(refresh_windows), int(cycles), int(warm_cycles))
    _check(load().kmc_set_electrostatics(h, C.byref(e)))


def kmc_solve_potential(h, r: int, ncell: int):
    phi = np.zeros(ncell, np.float64)
    res = C.c_double()
    _check(load().kmc_solve_potential(h, r, _ptr(phi), ncell, C.byref(res)))
    return phi, res.value


def kmc_read_potential_energy(h, r: int, nsite: int):
    u = np.zeros(nsite, np.int32)
    g = np.zeros((3, 8), np.int32)
    _check(load().kmc_read_potential_energy(h, r, _ptr(u), nsite, _ptr(g)))
    return u, g


def kmc_write_potential_energy(h, r: int, u, g=None):
    u = np.ascontiguousarray(u, np.int32)
    gp = None
    if g is not None:
        g = np.ascontiguousarray(g, np.int32)
        assert g.size == 24
        gp = _ptr(g)
    _check(load().kmc_write_potential_energy(h, r, _ptr(u), u.size, gp))


def kmc_set_grains(h, n_grains: int, width: int = 1, barrier_eV: float = 0.2):
    """Voronoi grains; n_grains <= 1 turns them off."""
    if n_grains <= 1:
        _check(load().kmc_set_grains(h, None))
        return
    g = kmc_grains(int(n_grains), int(width), float(barrier_eV))
    _check(load().kmc_set_grains(h, C.byref(g)))


def kmc_read_grains(h, r: int, ncell: int):
    grain = np.zeros(ncell, np.int32)
    bnd = np.zeros(ncell, np.uint8)
    _check(load().kmc_read_grains(h, r, _ptr(grain), _ptr(bnd), ncell))
    return grain, bnd


def kmc_read_dopants(h, r: int, ncell: int) -> np.ndarray:
    out = np.zeros(ncell, np.uint8)
    _check(load().kmc_read_dopants(h, r, _ptr(out), ncell))
    return out


def kmc_write_dopants(h, r: int, cells: np.ndarray):
    cells = np.ascontiguousarray(cells, np.uint8)
    _check(load().kmc_write_dopants(h, r, _ptr(cells), cells.size))


def kmc_read_site_field(h, r: int, nsite: int) -> np.ndarray:
    out = np.zeros(nsite, np.int32)
    _check(load().kmc_read_site_field(h, r, _ptr(out), nsite))
    return out


def kmc_destroy(h):
    _check(load().kmc_destroy(h))


def kmc_last_error() -> str:
    return load().kmc_last_error().decode()


# ------------------------------------------------------------ convenience
class TorchAllocator:
    """Device memory from torch's caching allocator for the ABI callback."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.live = {}
        self.c_alloc = kmc_alloc_fn(self._alloc)
        self.c_free = kmc_free_fn(self._free)

    def _alloc(self, ctx, nbytes):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # noqa: BLE001 - allocation failure is reported as NULL
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ctx, ptr):
        self.live.pop(ptr, None)


class Batch:
    """A batch of replicas (one lattice = a batch of one) on the current GPU."""

    def __init__(self, cells, comps, seed=0, *, edge=4, nfrag=None, precision=FKMC_PLAIN,
                 tracer=False, cap_v=0, n_tau=1.0, schedule=0, cluster_top=-1, small_pass=0, stream=None,
                 test_stuck_wait_us=0, alloc=None, lane_form=0, cluster_ctas=0):
        import torch
        self._alloc = TorchAllocator()
        o = kmc_default_opts()
        o.edge = int(edge)
        if nfrag is not None:
            for d in range(3):
                o.nfrag[d] = int(nfrag[d])
        o.precision = int(precision)
        o.tracer = int(bool(tracer))
        o.cap_v = int(cap_v)
        o.n_tau = float(n_tau)
        o.schedule = int(schedule)
        o.cluster_top = int(cluster_top)
        o.small_pass = int(small_pass)
        o.lane_form = int(lane_form)
        o.cluster_ctas = int(cluster_ctas)
        o.test_stuck_wait_us = int(test_stuck_wait_us)
        st = stream if stream is not None else torch.cuda.current_stream()
        o.stream = C.c_void_p(st.cuda_stream)
        if alloc is not None:  # an allocator of the caller's: an object with c_alloc / c_free callbacks
            self._alloc = alloc
        o.alloc = self._alloc.c_alloc
        o.free = self._alloc.c_free
        self._opts = o
        self.cells = [c if isinstance(c, kmc_cells) else kmc_cells(*c) for c in cells]
        # (n_vac, n_H) or (n_vac, n_H, n_Fe)
        self.comps = [c if isinstance(c, kmc_composition) else kmc_composition(*c) for c in comps]
        self.h = kmc_create_batch(self.cells, self.comps, seed, o)
        self.n = len(self.cells)

    def close(self):
        if getattr(self, "h", None):
            kmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def nsite(self, r=0):
        c = self.cells[r]
        return 3 * c.nx * c.ny * c.nz

    def set_barriers(self, Ea_O, Ea_H, T, prefactor=1e13, q_O=2.0, q_H=1.0, field_z=0.0):
        n = self.n
        bc = lambda v: np.broadcast_to(np.asarray(v, np.float64), (n,))  # noqa: E731
        EO, EH, A, qO, qH = bc(Ea_O), bc(Ea_H), bc(prefactor), bc(q_O), bc(q_H)
        tabs = [kmc_barrier_table(EO[i], EH[i], A[i], qO[i], qH[i]) for i in range(n)]
        kmc_set_barriers(self.h, tabs, bc(T), bc(field_z))

    def run(self, windows):
        return kmc_run(self.h, windows)

    def run_null(self, steps, n_frg):
        """The atom-based fragment kMC with null events (Sec. II.B)."""
        return kmc_run_null(self.h, steps, n_frg)

    def state(self, r=0):
        return kmc_read_state(self.h, r, self.nsite(r))

    def write_state(self, occ, r=0):
        kmc_write_state(self.h, r, occ)

    def records(self, r=0):
        return kmc_read_records(self.h, r)

    def tracer_field(self, r=0):
        return kmc_read_tracer(self.h, r, self.nsite(r))

    def moments(self, r=0, species=FKMC_V):
        return kmc_read_moments(self.h, r, species)

    def moments_all(self):
        return kmc_read_moments_all(self.h, self.n)

    def D(self, r=0, species=FKMC_V):
        return kmc_read_D(self.h, r, species)

    def info(self, r=0):
        return kmc_get_replica_info(self.h, r)

    def check(self, r=0):
        return kmc_check_invariants(self.h, r)

    def set_site_energy(self, vv=(), fe=()):
        kmc_set_site_energy(self.h, vv, fe)

    def set_electrostatics(self, eps_r=None, q_vac=2.0, refresh_windows=8, cycles=12, warm_cycles=0):
        kmc_set_electrostatics(self.h, eps_r, q_vac, refresh_windows, cycles, warm_cycles)

    def solve_potential(self, r=0):
        """(phi at every B node [z][y][x] flattened, relative residual)"""
        return kmc_solve_potential(self.h, r, self.nsite(r) // 3)

    def potential_energy(self, r=0):
        return kmc_read_potential_energy(self.h, r, self.nsite(r))

    def write_potential_energy(self, u, g=None, r=0):
        kmc_write_potential_energy(self.h, r, u, g)

    def set_grains(self, n_grains, width=1, barrier_eV=0.2):
        kmc_set_grains(self.h, n_grains, width, barrier_eV)

    def grains(self, r=0):
        return kmc_read_grains(self.h, r, self.nsite(r) // 3)

    def dopants(self, r=0):
        return kmc_read_dopants(self.h, r, self.nsite(r) // 3)

    def write_dopants(self, cells, r=0):
        kmc_write_dopants(self.h, r, cells)

    def site_field(self, r=0):
        return kmc_read_site_field(self.h, r, self.nsite(r))

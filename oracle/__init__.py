"""CPU oracle for the windowed fragment kMC (arXiv:2004.09081).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product path never
imports this package.  The oracle is plain serial C (``fkmc_oracle.c``),
compiled with ``-O2 -ffp-contract=off`` so that each floating-point operation is
one IEEE round-to-nearest operation, in source order.  It shares nothing with
the CUDA library.

Functions follow the paper: rates (Sec. II.A Eq. RateCnst1, Sec. III ESP term),
event selection (Eq. eventSelection), clock (Eq. TimeStep), fragment-local
selection (Sec. II.B Eq. AtomP), D from tracked trajectories (Sec. III),
site-energy interactions (Sec. "Oxygen vacancy diffusion with dopant and defect
interaction", Table add01).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fkmc_oracle.c")
_LIB = os.path.join(_HERE, "libfkmc_oracle.so")

SP_O, SP_H, SP_V = 0, 1, 2
PLAIN, MIXED = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, C99)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P, u64, i64, i32, u32, d = C.c_void_p, C.c_uint64, C.c_int64, C.c_int32, C.c_uint32, C.c_double
        sig = {
            "orc_philox4x64": (None, [P, P, P]),
            "orc_neglog64": (d, [u64]),
            "orc_neglog64_batch": (None, [P, P, i64]),
            "orc_partition_count": (C.c_int, [C.c_int, C.c_int]),
            "orc_neglog32": (C.c_float, [u64]),
            "orc_neighbour_table": (None, [P]),
            "orc_feistel": (u64, [u64, u64, u64, u32]),
            "orc_colour_perm": (None, [u64, u32, u64, P]),
            "orc_create": (P, [C.c_int] * 6 + [i64, i64, u64, u32, C.c_int]),
            "orc_destroy": (None, [P]),
            "orc_rate_table": (C.c_int, [d] * 8 + [C.c_int, P, P, P, P]),
            "orc_set_rates": (C.c_int, [P] + [d] * 8 + [C.c_int, d, C.c_int]),
            "orc_run": (C.c_int, [P, u64]),
            "orc_bkl_run": (C.c_int, [P, d, u64, P]),
            "orc_get_occ": (None, [P, P]),
            "orc_set_occ_records": (None, [P, P]),
            "orc_n_records": (i64, [P]),
            "orc_get_records": (i64, [P, P, i64]),
            "orc_get_tracer": (None, [P, P]),
            "orc_get_counters": (None, [P, P, P]),
            "orc_get_params": (None, [P, P, P, P]),
            "orc_moments": (C.c_int, [P, C.c_int, P]),
            "orc_place_dopants": (None, [P, i64]),
            "orc_set_dopants": (None, [P, P]),
            "orc_get_dopants": (C.c_int, [P, P]),
            "orc_set_site_energy": (C.c_int, [P, C.c_int, P, P, C.c_int, P, P]),
            "orc_site_shells": (C.c_int, [P, C.c_int, P, C.c_int]),
            "orc_site_energy": (i64, [P, i64, i64]),
            "orc_event_rate": (d, [P, i64, C.c_int]),
            "orc_null_pick": (u64, [u64, u64, u64, u32, u64]),
            "orc_null_run": (C.c_int, [P, u64, i64]),
            "orc_get_null": (None, [P, P, P, P, P]),
            "orc_set_grains": (C.c_int, [P, C.c_int, C.c_int, d]),
            "orc_set_elec": (C.c_int, [P, P, P]),
            "orc_get_grains": (None, [P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- primitives
def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def neglog64(x: int) -> float:
    return lib().orc_neglog64(int(x))


def neglog64_batch(x: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros(xs.size, np.float64)
    lib().orc_neglog64_batch(_ptr(xs), _ptr(out), xs.size)
    return out


def partition(cells, edge: int):
    """Fragments per dimension for a target fragment edge (even count nearest
    L/edge with edges >= 2 cells, else one fragment)."""
    return tuple(int(lib().orc_partition_count(int(L), int(edge))) for L in cells)


def neglog32(x: int) -> float:
    return lib().orc_neglog32(int(x))


def neighbour_table() -> np.ndarray:
    """int32 [3 types][8 neighbours][t2, dcx, dcy, dcz, dx, dy, dz]."""
    out = np.zeros((3, 8, 7), np.int32)
    lib().orc_neighbour_table(_ptr(out))
    return out


def feistel(i: int, nsite: int, seed: int, replica: int = 0) -> int:
    return int(lib().orc_feistel(i, nsite, seed, replica))


def colour_perm(seed: int, replica: int, w: int) -> np.ndarray:
    out = np.zeros(8, np.int32)
    lib().orc_colour_perm(seed, replica, w, _ptr(out))
    return out


def null_pick(p: int, n: int, seed: int, replica: int, step: int) -> int:
    return int(lib().orc_null_pick(p, n, seed, replica, step))


def rate_table(Ea_O, Ea_H, A, q_O, q_H, T, Ez, a_ang, cap_v=64):
    k64 = np.zeros(6, np.float64)
    k32 = np.zeros(6, np.float32)
    q = np.zeros(6, np.uint64)
    F = C.c_int32(0)
    rc = lib().orc_rate_table(Ea_O, Ea_H, A, q_O, q_H, T, Ez, a_ang, cap_v, _ptr(k64), _ptr(k32),
                              _ptr(q), C.byref(F))
    if rc:
        raise ValueError("bad rate parameters")
    return k64, k32, q, F.value


# ---------------------------------------------------------------- lattice
class Lattice:
    """One replica held by the oracle.  ``nf`` = fragments per dimension, or
    None to derive them from the target fragment edge ``edge`` (partition)."""

    def __init__(self, cells, nf, n_vac, n_H, seed=0, replica=0, tracer=False, n_Fe=0, edge=None):
        self.L = tuple(int(c) for c in cells)
        if nf is None:
            nf = partition(self.L, 4 if edge is None else edge)
        self.nf = tuple(int(f) for f in nf)
        self.nsite = 3 * self.L[0] * self.L[1] * self.L[2]
        self.ncell = self.L[0] * self.L[1] * self.L[2]
        self._h = lib().orc_create(*self.L, *self.nf, int(n_vac), int(n_H), int(seed), int(replica),
                                   int(bool(tracer)))
        if not self._h:
            raise ValueError("invalid lattice / partition / composition")
        self.tracer = bool(tracer)
        if n_Fe:
            lib().orc_place_dopants(self._h, int(n_Fe))

    # ---------------------------------------------- site-energy interactions
    def set_site_energy(self, vv=(), fe=()):
        """Shell energies: ``vv`` = [(d2, eV), ...] over O-O squared distances,
        ``fe`` = [(d2, eV), ...] over O-B squared distances, d2 in (a/2)^2."""
        vd = np.array([int(d) for d, _ in vv] or [0], np.int32)
        ve = np.array([float(e) for _, e in vv] or [0.0], np.float64)
        fd = np.array([int(d) for d, _ in fe] or [0], np.int32)
        fv = np.array([float(e) for _, e in fe] or [0.0], np.float64)
        rc = lib().orc_set_site_energy(self._h, len(vv), _ptr(vd), _ptr(ve), len(fe), _ptr(fd), _ptr(fv))
        if rc:
            raise ValueError("invalid site-energy shells for this lattice / partition / precision")

    def shells(self, t: int) -> np.ndarray:
        out = np.zeros((1024, 5), np.int32)
        k = lib().orc_site_shells(self._h, int(t), _ptr(out), 1024)
        return out[:k]

    def site_energy(self, s: int, exclude: int = -1) -> int:
        return int(lib().orc_site_energy(self._h, int(s), int(exclude)))

    def event_rate(self, s: int, n: int) -> float:
        return float(lib().orc_event_rate(self._h, int(s), int(n)))

    # ---------------------------------------------- null-event form (Sec. II.B)
    def null_run(self, steps: int, n_frg: int):
        """The atom-based fragment kMC with null events: `steps` steps of
        `n_frg` simultaneous vacancy picks."""
        if lib().orc_null_run(self._h, int(steps), int(n_frg)):
            raise RuntimeError("rates not set, site energies on, or bad n_frg")

    def null_clock(self):
        th, t = C.c_double(0), C.c_double(0)
        st = C.c_uint64(0)
        F = C.c_int32(0)
        lib().orc_get_null(self._h, C.byref(th), C.byref(t), C.byref(st), C.byref(F))
        return {"theta": th.value, "t": t.value, "steps": st.value, "F": F.value}

    # ---------------------------------------------- electrostatics (mu-scale model)
    def set_elec(self, u=None, g=None):
        """Frozen electrostatic field: u = rint(q phi 1e4) per O site and the
        self table g[3][8] (oracle/poisson.py); None turns it off."""
        if u is None:
            lib().orc_set_elec(self._h, None, None)
            return
        self._elec_u = np.ascontiguousarray(u, dtype=np.int32)
        self._elec_g = np.ascontiguousarray(g, dtype=np.int32)
        assert self._elec_u.size == self.nsite and self._elec_g.size == 24
        if lib().orc_set_elec(self._h, _ptr(self._elec_u), _ptr(self._elec_g)):
            raise ValueError("electrostatics need the plain form")

    # ---------------------------------------------- grains (mu-scale model)
    def set_grains(self, n_grains: int, width: int = 1, barrier_eV: float = 0.2):
        """Voronoi grains; hops touching a boundary cell get barrier + barrier_eV."""
        if lib().orc_set_grains(self._h, int(n_grains), int(width), float(barrier_eV)):
            raise ValueError("invalid grain parameters for this lattice")

    def grains(self):
        g = np.zeros(self.ncell, np.int32)
        bnd = np.zeros(self.ncell, np.uint8)
        lib().orc_get_grains(self._h, _ptr(g), _ptr(bnd))
        return g, bnd

    def dopants(self) -> np.ndarray:
        out = np.zeros(self.ncell, np.uint8)
        lib().orc_get_dopants(self._h, _ptr(out))
        return out

    def set_dopants(self, cells: np.ndarray):
        cells = np.ascontiguousarray(cells, dtype=np.uint8)
        assert cells.size == self.ncell
        lib().orc_set_dopants(self._h, _ptr(cells))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_rates(self, Ea_O, Ea_H, T, A=1e13, q_O=2.0, q_H=1.0, Ez=0.0, a_ang=3.905, cap_v=64,
                  n_tau=1.0, precision=PLAIN):
        rc = lib().orc_set_rates(self._h, Ea_O, Ea_H, A, q_O, q_H, T, Ez, a_ang, cap_v, n_tau,
                                 precision)
        if rc:
            raise ValueError("bad rate parameters")
        self.a_ang = a_ang

    def run(self, windows: int):
        if lib().orc_run(self._h, int(windows)):
            raise RuntimeError("rates not set")

    def bkl_run(self, t_end: float, stream: int = 0) -> float:
        t = C.c_double(0)
        if lib().orc_bkl_run(self._h, float(t_end), int(stream), C.byref(t)):
            raise RuntimeError("rates not set")
        return t.value

    def occupancy(self) -> np.ndarray:
        out = np.zeros(self.nsite, np.uint8)
        lib().orc_get_occ(self._h, _ptr(out))
        return out

    def set_occupancy(self, occ: np.ndarray):
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        assert occ.size == self.nsite
        lib().orc_set_occ_records(self._h, _ptr(occ))

    def records(self) -> np.ndarray:
        n = lib().orc_n_records(self._h)
        out = np.zeros((max(n, 1), 6), np.int64)
        k = lib().orc_get_records(self._h, _ptr(out), n)
        return out[:k]

    def tracer_field(self) -> np.ndarray:
        out = np.zeros((self.nsite, 3), np.int32)
        lib().orc_get_tracer(self._h, _ptr(out))
        return out

    def counters(self):
        c = np.zeros(3, np.uint64)
        cs = C.c_double(0)
        lib().orc_get_counters(self._h, _ptr(c), C.byref(cs))
        return {"window": int(c[0]), "hops": int(c[1]), "handoffs": int(c[2]),
                "clock_sum": cs.value}

    def params(self):
        tau, th = C.c_double(0), C.c_double(0)
        F = C.c_int32(0)
        lib().orc_get_params(self._h, C.byref(tau), C.byref(th), C.byref(F))
        return {"tau": tau.value, "theta_tau": th.value, "F": F.value}

    def moments(self, species=SP_V) -> np.ndarray:
        out = np.zeros(7, np.int64)
        if lib().orc_moments(self._h, int(species), _ptr(out)):
            raise RuntimeError("tracer field not enabled")
        return out

    def diffusion(self, species=SP_V, t=None):
        """D of one species from its tracked displacements (Sec. III, D from
        per-atom trajectories); see diffusion_from_moments."""
        m = self.moments(species)
        if t is None:
            t = self.counters()["window"] * self.params()["tau"] + self.null_clock()["t"]
        return diffusion_from_moments(m, t, self.a_ang)


def diffusion_from_moments(m, t: float, a_ang: float):
    """D from the integer moments m = {count, sum d_k, sum d_k^2} (units a/2)
    after time t (s), a in Angstrom; every mean is over the tracked particles:
      D      = (<dx^2> + <dy^2> + <dz^2>) / (6 t)        mean squared displacement
      D_xy   = (<dx^2> + <dy^2>) / (4 t)                 in-plane
      D_axes = (<d_k^2> - <d_k>^2) / (2 t)               per axis, drift removed
      D_z    = D_axes[2]                                 along the field
      v      = <d_k> / t                                 drift velocity
    Moments of several independent lattices may be summed first (pooled)."""
    m = np.asarray(m, dtype=np.int64)
    n = max(int(m[0]), 1)
    h = 0.5 * a_ang * 1e-10
    msd = m[4:7].astype(np.float64) / n * h * h
    mean = m[1:4].astype(np.float64) / n * h
    var = msd - mean * mean
    return {"D": msd.sum() / (6 * t), "D_xy": (msd[0] + msd[1]) / (4 * t), "D_axes": var / (2 * t),
            "D_z": var[2] / (2 * t), "v": mean / t, "msd": msd, "mean": mean, "t": t, "n": n}

"""Oracle for the fractional-step parallel KMC method (test infrastructure).

A plain, slow CPU restatement of what the CUDA library computes, written
from the paper (Arampatzis, Katsoulakis, Plechac, Taufer, Xu,
"Hierarchical fractional-step approximations and parallel kinetic Monte
Carlo algorithms"). It is the yardstick for the CUDA path, never part of it:
only the tests, the smoke check and the benchmark's CPU baseline may import
this package. It shares no code with ``paper_1105_4673_gb300``.

Parts:
  * ``fskmc_oracle.c`` (loaded here through ctypes): Philox4x32-10, rate
    classes, the FS window SSA cell by cell, the schedules, the serial SSA,
    integer observables.
  * ``brute.py``: exact generator matrices and operator products on tiny
    lattices (numpy / scipy).
  * ``closed_forms.py``: the closed forms the paper prints or implies.

Parity: every function here is pinned by a test under ``tests/`` against
something other than itself (see ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fskmc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

MODELS = {"ADSDES": 0, "ISING": 1, "DIFFUSION": 2, "ZGB": 3, "ISING1D": 4}
SCHEMES = {"LIE": 0, "STRANG": 1, "RANDOM": 2, "RANDOM_ORDER": 3}
NCLASS = {0: 10, 1: 10, 2: 15, 3: 4, 4: 6}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-adds) and return the path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-pthread", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        L.orc_philox.argtypes = [u32p, u32p, u32p]
        L.orc_rates.argtypes = [C.c_int] + [C.c_double] * 7 + [f64p]
        L.orc_rates.restype = C.c_int
        L.orc_init_bernoulli.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_double, C.c_uint32, u8p]
        L.orc_init_bump.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_double, C.c_double,
                                    C.c_int, C.c_uint32, u8p]
        L.orc_schedule.argtypes = [C.c_int, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                   C.c_uint32, C.c_void_p, C.c_void_p, C.c_int64]
        L.orc_schedule.restype = C.c_int64
        L.orc_fs_run.argtypes = [C.c_int] * 5 + [f64p, C.c_int, C.c_double, C.c_double,
                                                 C.c_uint64, C.c_uint32, u32p, C.c_int, u8p,
                                                 u64p, C.c_void_p]
        L.orc_fs_run.restype = C.c_int
        L.orc_window.argtypes = [C.c_int] * 5 + [f64p, C.c_int, C.c_double, C.c_uint32,
                                                 C.c_uint64, C.c_uint32, u8p, u64p,
                                                 C.c_void_p, C.c_void_p]
        L.orc_window.restype = C.c_int
        L.orc_ssa_run.argtypes = [C.c_int, C.c_int, C.c_int, f64p, C.c_double, C.c_uint64,
                                  C.c_uint32, u8p]
        L.orc_ssa_run.restype = C.c_int64
        L.orc_ssa_bkl_run.argtypes = [C.c_int, C.c_int, C.c_int, f64p, C.c_double, C.c_uint64,
                                      C.c_uint32, u8p]
        L.orc_ssa_bkl_run.restype = C.c_int64
        L.orc_total_rate.argtypes = [C.c_int, C.c_int, C.c_int, f64p, u8p, i64p]
        L.orc_total_rate.restype = C.c_double
        L.orc_cell_members.argtypes = [C.c_int] * 5 + [f64p, u8p, C.c_int, C.c_int,
                                                       i32p, i32p, i32p, i32p]
        L.orc_cell_members.restype = C.c_int
        L.orc_cell_writeset.argtypes = [C.c_int] * 7 + [i32p]
        L.orc_cell_writeset.restype = C.c_int
        L.orc_observables.argtypes = [C.c_int, C.c_int, u8p, C.c_int, i64p, i64p, i64p, i64p]
        L.orc_fs_ensemble.argtypes = [C.c_int] * 5 + [f64p, C.c_int, C.c_double, C.c_double,
                                                      C.c_uint64, C.c_int, u8p, u8p]
        L.orc_fs_ensemble.restype = C.c_int
        L.orc_ssa_ensemble.argtypes = [C.c_int, C.c_int, C.c_int, f64p, C.c_double, C.c_uint64,
                                       C.c_int, u8p, u8p]
        L.orc_ssa_ensemble.restype = C.c_int
        L.orc_window_cells.argtypes = [C.c_int] * 5 + [f64p, C.c_int, C.c_double, C.c_uint32,
                                                       C.c_uint64, C.c_uint32, u8p, C.c_int, i32p,
                                                       i32p, i32p]
        L.orc_window_cells.restype = C.c_int
        L.orc_fs_run_threads.argtypes = [C.c_int] * 5 + [f64p, C.c_int, C.c_double, C.c_double,
                                                         C.c_uint64, C.c_uint32, u32p, u8p, u64p,
                                                         C.c_void_p, C.c_int]
        L.orc_fs_run_threads.restype = C.c_int
        L.orc_fs2_run.argtypes = [C.c_int] * 7 + [f64p, C.c_int, C.c_double, C.c_double, C.c_int,
                                                  C.c_int, C.c_uint64, C.c_uint32, u32p, u8p, u64p,
                                                  C.c_void_p]
        L.orc_fs2_run.restype = C.c_int
        L.orc_fs2_ensemble.argtypes = [C.c_int] * 7 + [f64p, C.c_int, C.c_double, C.c_double,
                                                       C.c_int, C.c_int, C.c_uint64, C.c_int, u8p,
                                                       u8p]
        L.orc_fs2_ensemble.restype = C.c_int
        _lib = L
    return _lib


def _rates6(rates: dict) -> np.ndarray:
    """{ka, kd, betaJ, nu, yA, kr, betah} as the C side reads them."""
    return np.array([rates.get("ka", 1.0), rates.get("kd", 1.0), rates.get("betaJ", 0.0),
                     rates.get("nu", 0.0), rates.get("yA", 0.0), rates.get("kr", 0.0),
                     rates.get("betah", 0.0)], dtype=np.float64)


def _model(model) -> int:
    return MODELS[model] if isinstance(model, str) else int(model)


def _scheme(scheme) -> int:
    return SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def rates(model, **kw) -> np.ndarray:
    """Class rates r_k in class order (see orc_rates in fskmc_oracle.c)."""
    r = np.zeros(16, np.float64)
    m = _model(model)
    n = lib().orc_rates(m, *_rates6(kw), r)
    return r[:n]


def init_bernoulli(lx: int, ly: int, seed: int, p: float, replica: int = 0) -> np.ndarray:
    lat = np.zeros(lx * ly, np.uint8)
    lib().orc_init_bernoulli(lx, ly, seed, p, replica, lat)
    return lat


def init_bump(lx: int, ly: int, seed: int, amp: float, width: float, species: int = 1,
              replica: int = 0) -> np.ndarray:
    lat = np.zeros(lx * ly, np.uint8)
    lib().orc_init_bump(lx, ly, seed, amp, width, species, replica, lat)
    return lat


def schedule(scheme, dt: float, T: float, seed: int = 0, replica: int = 0, w0: int = 0):
    """(colours, lengths) of the windows of a run; colour 0 = E, 1 = O."""
    s = _scheme(scheme)
    n = lib().orc_schedule(s, dt, T, seed, replica, w0, None, None, 0)
    if n < 0:
        raise ValueError("invalid schedule arguments")
    col = np.zeros(max(n, 1), np.int32)
    h = np.zeros(max(n, 1), np.float64)
    lib().orc_schedule(s, dt, T, seed, replica, w0, col.ctypes.data, h.ctypes.data, n)
    return col[:n], h[:n]


class FSRun:
    """Stateful FS run on one lattice (the oracle's counterpart of a context)."""

    def __init__(self, lx, ly, qx, qy, model, rates: dict, lattice=None, replica: int = 0):
        self.lx, self.ly, self.qx, self.qy = lx, ly, qx, qy
        self.model = _model(model)
        self.r6 = _rates6(rates)
        self.replica = replica
        self.lat = (np.zeros(lx * ly, np.uint8) if lattice is None
                    else np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1).copy())
        self.w = np.zeros(1, np.uint32)
        self.stats = np.zeros(3, np.uint64)
        self.workload = np.zeros((lx // qx) * (ly // qy), np.int32)

    def run(self, scheme, dt, T, seed, order: int = 0):
        rc = lib().orc_fs_run(self.lx, self.ly, self.qx, self.qy, self.model, self.r6,
                              _scheme(scheme), dt, T, seed, self.replica, self.w, order,
                              self.lat, self.stats, self.workload.ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the run arguments")
        return self

    def run_threads(self, scheme, dt, T, seed, nthreads: int):
        """The same run with each window's cells spread over nthreads threads
        (bit-identical to run(): same-colour cells are independent)."""
        rc = lib().orc_fs_run_threads(self.lx, self.ly, self.qx, self.qy, self.model, self.r6,
                                      _scheme(scheme), dt, T, seed, self.replica, self.w, self.lat,
                                      self.stats, self.workload.ctypes.data, nthreads)
        if rc != 0:
            raise ValueError("oracle rejected the run arguments")
        return self

    def window(self, colour: int, h: float, seed: int, w: int | None = None):
        """One window; returns per-cell ambiguous flags."""
        amb = np.zeros_like(self.workload)
        ww = int(self.w[0]) if w is None else w
        rc = lib().orc_window(self.lx, self.ly, self.qx, self.qy, self.model, self.r6,
                              colour, h, ww, seed, self.replica, self.lat, self.stats,
                              self.workload.ctypes.data, amb.ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the window arguments")
        self.w[0] = ww + 1
        return amb

    @property
    def events(self) -> int:
        return int(self.stats[0])

    @property
    def windows(self) -> int:
        return int(self.stats[1])

    @property
    def ambiguous(self) -> int:
        return int(self.stats[2])


class FS2Run:
    """Nested (two-level) FS run on one lattice, Section 5 (Eq. sublatt2,
    Eq. opdecomp2): super-cells Qx x Qy in a checkerboard, each a
    checkerboard of sub-cells qx x qy; the outer schedule over super-cell
    colours, n_in inner steps of the inner schedule (LIE or STRANG) over the
    sub-cell colours inside every outer window. Spin-flip models only."""

    def __init__(self, lx, ly, Q, q, model, rates: dict, lattice=None, replica: int = 0):
        self.lx, self.ly = lx, ly
        self.Qx, self.Qy = Q
        self.qx, self.qy = q
        self.model = _model(model)
        self.r6 = _rates6(rates)
        self.replica = replica
        self.lat = (np.zeros(lx * ly, np.uint8) if lattice is None
                    else np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1).copy())
        self.w = np.zeros(1, np.uint32)
        self.stats = np.zeros(3, np.uint64)
        self.workload = np.zeros((lx // self.qx) * (ly // self.qy), np.int32)

    def run(self, scheme, dt, T, seed, inner="LIE", n_in: int = 1):
        rc = lib().orc_fs2_run(self.lx, self.ly, self.Qx, self.Qy, self.qx, self.qy, self.model,
                               self.r6, _scheme(scheme), dt, T, _scheme(inner), n_in, seed,
                               self.replica, self.w, self.lat, self.stats,
                               self.workload.ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the nested run arguments")
        return self

    @property
    def events(self) -> int:
        return int(self.stats[0])

    @property
    def windows(self) -> int:
        return int(self.stats[1])

    @property
    def ambiguous(self) -> int:
        return int(self.stats[2])


def fs2_ensemble(lx, ly, Q, q, model, rates: dict, scheme, dt, T, seed, M, init, inner="LIE",
                 n_in: int = 1) -> np.ndarray:
    """Final states (M, lx*ly) of M independent nested runs (replicas 0..M-1)."""
    init = np.ascontiguousarray(init, dtype=np.uint8).reshape(-1)
    out = np.zeros((M, lx * ly), np.uint8)
    rc = lib().orc_fs2_ensemble(lx, ly, Q[0], Q[1], q[0], q[1], _model(model), _rates6(rates),
                                _scheme(scheme), dt, T, _scheme(inner), n_in, seed, M, init,
                                out.reshape(-1))
    if rc != 0:
        raise ValueError("oracle rejected the ensemble arguments")
    return out


def ssa_run(lx, ly, model, rates: dict, lattice, T: float, seed: int, replica: int = 0):
    """Serial SSA over the whole lattice; returns (lattice, events)."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1).copy()
    n = lib().orc_ssa_run(lx, ly, _model(model), _rates6(rates), T, seed, replica, lat)
    if n < 0:
        raise ValueError("oracle rejected the SSA arguments")
    return lat, int(n)


def ssa_bkl_run(lx, ly, model, rates: dict, lattice, T: float, seed: int, replica: int = 0):
    """Serial SSA with class lists (the BKL form); returns (lattice, events)."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1).copy()
    n = lib().orc_ssa_bkl_run(lx, ly, _model(model), _rates6(rates), T, seed, replica, lat)
    if n < 0:
        raise ValueError("oracle rejected the SSA arguments")
    return lat, int(n)


def total_rate(lx, ly, model, rates: dict, lattice):
    counts = np.zeros(16, np.int64)
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1)
    lam = lib().orc_total_rate(lx, ly, _model(model), _rates6(rates), lat, counts)
    return lam, counts[:NCLASS[_model(model)]]


def cell_members(lx, ly, qx, qy, model, rates: dict, lattice, m: int, colour: int):
    cap = 9 * qx * qy + 8
    o, t, k, c = (np.zeros(cap, np.int32) for _ in range(4))
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1)
    n = lib().orc_cell_members(lx, ly, qx, qy, _model(model), _rates6(rates), lat, m, colour,
                               o, t, k, c)
    return o[:n], t[:n], k[:n], c[:n]


def cell_writeset(lx, ly, qx, qy, model, m: int, colour: int) -> np.ndarray:
    out = np.zeros(qx * qy + 2 * (qx + qy) + 8, np.int32)
    n = lib().orc_cell_writeset(lx, ly, qx, qy, _model(model), m, colour, out)
    return out[:n]


def observables_int(lx, ly, lattice, rmax: int):
    """(counts[3], pairs, gx[rmax], gy[rmax]) as exact integers."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1)
    counts = np.zeros(3, np.int64)
    pairs = np.zeros(1, np.int64)
    gx = np.zeros(max(rmax, 1), np.int64)
    gy = np.zeros(max(rmax, 1), np.int64)
    lib().orc_observables(lx, ly, lat, rmax, counts, pairs, gx, gy)
    return counts, int(pairs[0]), gx[:rmax], gy[:rmax]


def observables(lx, ly, model, lattice, rmax: int):
    """Coverage per state, energy per site and pair correlations (Section 7).

    energy: -(occupied nearest-neighbour pairs)/N for the lattice-gas models,
    -(1/N) sum_<xy> s_x s_y with s = 2 sigma - 1 for ISING, NaN for ZGB.
    paircorr: [G_x(1..rmax), G_y(1..rmax)], G_e(r) = (1/N) sum_x
    [sigma(x)=1][sigma(x+r e)=1].
    """
    m = _model(model)
    N = lx * ly
    counts, pairs, gx, gy = observables_int(lx, ly, lattice, rmax)
    cov = counts / N
    if m == 3:
        energy = float("nan")
    elif m == 1:
        energy = -(4.0 * pairs - 8.0 * counts[1] + 2.0 * N) / N
    else:
        energy = -pairs / N
    pc = np.concatenate([gx, gy]).astype(np.float64) / N
    return cov, energy, pc


def fs_ensemble(lx, ly, qx, qy, model, rates: dict, scheme, dt, T, seed, M, init) -> np.ndarray:
    """Final states (M, lx*ly) of M independent FS runs (replicas 0..M-1)."""
    init = np.ascontiguousarray(init, dtype=np.uint8).reshape(-1)
    out = np.zeros((M, lx * ly), np.uint8)
    rc = lib().orc_fs_ensemble(lx, ly, qx, qy, _model(model), _rates6(rates), _scheme(scheme),
                               dt, T, seed, M, init, out.reshape(-1))
    if rc != 0:
        raise ValueError("oracle rejected the ensemble arguments")
    return out


def ssa_ensemble(lx, ly, model, rates: dict, T, seed, M, init) -> np.ndarray:
    """Final states (M, lx*ly) of M independent serial SSA runs."""
    init = np.ascontiguousarray(init, dtype=np.uint8).reshape(-1)
    out = np.zeros((M, lx * ly), np.uint8)
    rc = lib().orc_ssa_ensemble(lx, ly, _model(model), _rates6(rates), T, seed, M, init,
                                out.reshape(-1))
    if rc != 0:
        raise ValueError("oracle rejected the ensemble arguments")
    return out


def window_cells(lx, ly, qx, qy, model, rates: dict, lattice, colour: int, h: float, w: int,
                 seed: int, cells, replica: int = 0):
    """One window for the listed cells only; returns (lattice after, events, ambiguous)."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1).copy()
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    ev = np.zeros(len(cells), np.int32)
    amb = np.zeros(len(cells), np.int32)
    rc = lib().orc_window_cells(lx, ly, qx, qy, _model(model), _rates6(rates), colour, h, w, seed,
                                replica, lat, len(cells), cells, ev, amb)
    if rc != 0:
        raise ValueError("oracle rejected the window arguments")
    return lat, ev, amb

"""GB300 fractional-step parallel kinetic Monte Carlo (thin Python binding).

Argument marshalling over the C ABI of ``include/fskmc.h`` (libfskmc.so,
built in-tree by ``paper_1105_4673_gb300.build``). Every step of the method
runs in the library's CUDA kernels; there is no Python or CPU fallback: if
the library is missing this module raises on first use.

The functions below carry the C names; ``Context`` wraps a context handle
for convenience. Lattices cross the boundary as uint8 numpy arrays (host) or
as CUDA tensors / raw device pointers (device); PyTorch is used only for
device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfskmc.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(6)
MODELS = {"ADSDES": 0, "ISING": 1, "ISING_ARRHENIUS": 1, "DIFFUSION": 2, "ADSDES_DIFFUSION": 2,
          "ZGB": 3, "ISING1D": 4}
SCHEMES = {"LIE": 0, "STRANG": 1, "RANDOM": 2, "RANDOM_ORDER": 3}
CLOCKS = {"FP64": 0, "FP32": 1}
ENGINES = {"PLAIN": 0, "PERSISTENT": 1}
ORDERS = {"NATURAL": 0, "WORKLOAD": 1, "AUTO": 2}
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESTATE"}

# Every entry point the header declares (checked by the tests).
EXPORTS = [
    "fskmc_create", "fskmc_batch_create", "fskmc_destroy", "fskmc_last_error",
    "fskmc_set_replica_id", "fskmc_set_clock", "fskmc_set_engine", "fskmc_set_warps_per_block",
    "fskmc_set_cell_grouping", "fskmc_set_edge_screen", "fskmc_set_spin_limit", "fskmc_set_task_order", "fskmc_info", "fskmc_init_random", "fskmc_init_bump",
    "fskmc_set_state", "fskmc_get_state", "fskmc_state_layout", "fskmc_set_state_all", "fskmc_get_state_all",
    "fskmc_run", "fskmc_window", "fskmc_get_window_index",
    "fskmc_set_window_index", "fskmc_observables", "fskmc_stats", "fskmc_exact_edge_checks", "fskmc_workload", "fskmc_sync",
    "fskmc_observables_noalloc", "fskmc_autotune", "fskmc_selftest_divide", "fskmc_selftest_log",
    "fskmc_schedule", "fskmc_set_nesting",
]
NOALLOC_MAX_RMAX = 256


class FskmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Lattice(C.Structure):
    _fields_ = [("lx", C.c_int32), ("ly", C.c_int32), ("bitpacked", C.c_int32)]


class Rates(C.Structure):
    _fields_ = [("ka", C.c_double), ("kd", C.c_double), ("betaJ", C.c_double),
                ("nu", C.c_double), ("yA", C.c_double), ("kr", C.c_double),
                ("betah", C.c_double)]


class CellShape(C.Structure):
    _fields_ = [("qx", C.c_int32), ("qy", C.c_int32)]


_lib = None


def lib():
    """Load libfskmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfskmc.so not built ({LIB_PATH}); run "
                              "`python -m paper_1105_4673_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, u8p = C.c_void_p, C.POINTER(C.c_uint8)
        sig = {
            "fskmc_create": ([C.POINTER(Lattice), C.c_int, C.POINTER(Rates), CellShape, vp,
                              C.POINTER(vp)], C.c_int),
            "fskmc_batch_create": ([C.c_int32, C.POINTER(Lattice), C.c_int, C.POINTER(Rates),
                                    CellShape, vp, C.POINTER(vp)], C.c_int),
            "fskmc_destroy": ([vp], None),
            "fskmc_last_error": ([vp], C.c_char_p),
            "fskmc_set_replica_id": ([vp, C.c_uint32], C.c_int),
            "fskmc_set_clock": ([vp, C.c_int], C.c_int),
            "fskmc_set_engine": ([vp, C.c_int], C.c_int),
            "fskmc_set_warps_per_block": ([vp, C.c_int32], C.c_int),
            "fskmc_set_cell_grouping": ([vp, C.c_int32], C.c_int),
            "fskmc_set_edge_screen": ([vp, C.c_int32], C.c_int),
            "fskmc_set_spin_limit": ([vp, C.c_uint32], C.c_int),
            "fskmc_set_task_order": ([vp, C.c_int], C.c_int),
            "fskmc_set_nesting": ([vp, CellShape, C.c_int, C.c_int32], C.c_int),
            "fskmc_info": ([vp, C.POINTER(C.c_int32)], C.c_int),
            "fskmc_init_random": ([vp, C.c_uint64, C.c_double], C.c_int),
            "fskmc_init_bump": ([vp, C.c_uint64, C.c_double, C.c_double, C.c_int32], C.c_int),
            "fskmc_set_state": ([vp, C.c_int32, vp, C.c_int32], C.c_int),
            "fskmc_get_state": ([vp, C.c_int32, vp, C.c_int32], C.c_int),
            "fskmc_state_layout": ([vp, C.POINTER(C.c_int64)], C.c_int),
            "fskmc_set_state_all": ([vp, vp, C.c_int32], C.c_int),
            "fskmc_get_state_all": ([vp, vp, C.c_int32], C.c_int),
            "fskmc_run": ([vp, C.c_int, C.c_double, C.c_double, C.c_uint64], C.c_int),
            "fskmc_window": ([vp, C.c_int32, C.c_double, C.c_uint64], C.c_int),
            "fskmc_get_window_index": ([vp, C.POINTER(C.c_uint64)], C.c_int),
            "fskmc_set_window_index": ([vp, C.c_uint64], C.c_int),
            "fskmc_observables": ([vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.c_int32], C.c_int),
            "fskmc_stats": ([vp, C.POINTER(C.c_uint64)], C.c_int),
            "fskmc_exact_edge_checks": ([vp, C.POINTER(C.c_uint64)], C.c_int),
            "fskmc_workload": ([vp, C.c_int32, C.POINTER(C.c_int32)], C.c_int),
            "fskmc_sync": ([vp], C.c_int),
            "fskmc_selftest_divide": ([vp, vp, C.c_int32, C.POINTER(C.c_uint32)], C.c_int),
            "fskmc_selftest_log": ([vp, C.c_int32, vp], C.c_int),
            "fskmc_schedule": ([C.c_int, C.c_double, C.c_double, C.c_uint64, C.c_uint32, C.c_uint64,
                                vp, vp, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
            "fskmc_autotune": ([C.c_int32, C.POINTER(Lattice), C.c_int, C.POINTER(Rates), C.c_int,
                                C.c_double, C.c_int, C.c_int, C.c_double, C.c_uint64, vp,
                                C.POINTER(CellShape), C.POINTER(C.c_int32),
                                C.POINTER(C.c_double)], C.c_int),
            "fskmc_observables_noalloc": ([vp, C.c_int32, C.c_int32, C.c_int, vp,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.c_int32], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        del u8p
        _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != OK:
        msg = lib().fskmc_last_error(ctx)
        raise FskmcError(status, msg.decode() if msg else "")


def _rates(d: dict) -> Rates:
    return Rates(d.get("ka", 1.0), d.get("kd", 1.0), d.get("betaJ", 0.0), d.get("nu", 0.0),
                 d.get("yA", 0.0), d.get("kr", 0.0), d.get("betah", 0.0))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


def _ptr_of(buf):
    """(pointer, is_device) of a numpy array, a CUDA tensor or a raw int."""
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("lattice arrays must be C-contiguous uint8")
        return buf.ctypes.data, 0
    if hasattr(buf, "data_ptr"):
        if buf.dtype.__repr__() != "torch.uint8" or not buf.is_contiguous():
            raise ValueError("lattice tensors must be contiguous uint8")
        return buf.data_ptr(), 1 if buf.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


class Context:
    """One library context (a single lattice or a batch of replicas)."""

    def __init__(self, lx=None, ly=None, model="ADSDES", rates=None, q=(8, 8), stream=None,
                 batch=None, bitpacked=False):
        L = lib()
        h = C.c_void_p()
        m = MODELS[model] if isinstance(model, str) else int(model)
        shape = CellShape(*(q if q is not None else (0, 0)))
        if batch is None:
            self.sizes = [(lx, ly)]
            st = L.fskmc_create(C.byref(Lattice(lx, ly, int(bitpacked))), m, C.byref(_rates(rates or {})),
                                shape, _stream_ptr(stream), C.byref(h))
        else:
            n = len(batch)
            lats = (Lattice * n)(*[Lattice(b["lx"], b["ly"], int(bitpacked)) for b in batch])
            rts = (Rates * n)(*[_rates(b["rates"]) for b in batch])
            self.sizes = [(b["lx"], b["ly"]) for b in batch]
            st = L.fskmc_batch_create(n, lats, m, rts, shape, _stream_ptr(stream), C.byref(h))
        _check(st)
        self.h = h
        self.model = m

    def close(self):
        if getattr(self, "h", None):
            lib().fskmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration ----------------------------------------------------
    def set_replica_id(self, r: int):
        _check(lib().fskmc_set_replica_id(self.h, r), self.h)

    def set_clock(self, clock):
        _check(lib().fskmc_set_clock(self.h, CLOCKS[clock] if isinstance(clock, str) else clock), self.h)

    def set_engine(self, engine):
        _check(lib().fskmc_set_engine(self.h, ENGINES[engine] if isinstance(engine, str) else engine),
               self.h)

    def set_warps_per_block(self, w: int):
        _check(lib().fskmc_set_warps_per_block(self.h, w), self.h)

    def set_cell_grouping(self, mode):
        """True / False / "AUTO" (the library default)."""
        m = 2 if mode == "AUTO" else (1 if mode else 0)
        _check(lib().fskmc_set_cell_grouping(self.h, m), self.h)

    def set_edge_screen(self, on: bool):
        """Binary64 clock: screened window-edge decisions (True, the default)
        or every decision from the binary64 divide (False)."""
        _check(lib().fskmc_set_edge_screen(self.h, 1 if on else 0), self.h)

    def set_spin_limit(self, polls: int):
        _check(lib().fskmc_set_spin_limit(self.h, polls), self.h)

    def set_task_order(self, order):
        o = ORDERS[order] if isinstance(order, str) else int(order)
        _check(lib().fskmc_set_task_order(self.h, o), self.h)

    def set_nesting(self, super_cell, inner="LIE", n_inner: int = 1):
        """Nested two-level scheme (Section 5): super-cells of shape
        super_cell, each a checkerboard of the context's cells, with n_inner
        inner steps of the inner schedule per outer window; None turns it
        off."""
        shape = CellShape(*(super_cell if super_cell else (0, 0)))
        s = SCHEMES[inner] if isinstance(inner, str) else int(inner)
        _check(lib().fskmc_set_nesting(self.h, shape, s, n_inner), self.h)

    def info(self) -> dict:
        out = (C.c_int32 * 6)()
        _check(lib().fskmc_info(self.h, out), self.h)
        return dict(qx=out[0], qy=out[1], replicas=out[2], cells=out[3], warps_per_block=out[4],
                    lanes_per_cell=out[5])

    # -- state -----------------------------------------------------------
    def init_random(self, seed: int, coverage: float):
        _check(lib().fskmc_init_random(self.h, seed, coverage), self.h)

    def init_bump(self, seed: int, amp: float, width: float, species: int = 1):
        _check(lib().fskmc_init_bump(self.h, seed, amp, width, species), self.h)

    def set_state(self, lattice, replica: int = 0):
        if isinstance(lattice, np.ndarray):
            lattice = np.ascontiguousarray(lattice, dtype=np.uint8).reshape(-1)
        p, dev = _ptr_of(lattice)
        _check(lib().fskmc_set_state(self.h, replica, p, dev), self.h)

    def get_state(self, replica: int = 0, out=None) -> np.ndarray:
        lx, ly = self.sizes[replica]
        if out is None:
            out = np.empty(lx * ly, np.uint8)
        p, dev = _ptr_of(out)
        _check(lib().fskmc_get_state(self.h, replica, p, dev), self.h)
        return out

    def state_layout(self) -> np.ndarray:
        """Byte offset of every replica's lattice in the batch's state buffer,
        then the buffer's size (fskmc_state_layout)."""
        out = (C.c_int64 * (len(self.sizes) + 1))()
        _check(lib().fskmc_state_layout(self.h, out), self.h)
        return np.array(out[:], np.int64)

    def set_state_all(self, buf):
        """Every replica's lattice in one copy, from a buffer in the layout of
        state_layout() (host array, or a CUDA tensor)."""
        if isinstance(buf, np.ndarray):
            buf = np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
        p, dev = _ptr_of(buf)
        _check(lib().fskmc_set_state_all(self.h, p, dev), self.h)

    def get_state_all(self, out=None):
        """Every replica's lattice in one copy, in the layout of state_layout()."""
        if out is None:
            out = np.empty(int(self.state_layout()[-1]), np.uint8)
        p, dev = _ptr_of(out)
        _check(lib().fskmc_get_state_all(self.h, p, dev), self.h)
        return out

    # -- the method --------------------------------------------------------
    def run(self, scheme, dt: float, T: float, seed: int):
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        _check(lib().fskmc_run(self.h, s, dt, T, seed), self.h)

    def window(self, colour: int, h: float, seed: int):
        _check(lib().fskmc_window(self.h, colour, h, seed), self.h)

    @property
    def window_index(self) -> int:
        w = C.c_uint64()
        _check(lib().fskmc_get_window_index(self.h, C.byref(w)), self.h)
        return w.value

    @window_index.setter
    def window_index(self, w: int):
        _check(lib().fskmc_set_window_index(self.h, w), self.h)

    def observables(self, replica: int = 0, rmax: int = 0):
        cov = (C.c_double * 3)()
        en = C.c_double()
        pc = (C.c_double * max(2 * rmax, 1))()
        _check(lib().fskmc_observables(self.h, replica, cov, C.byref(en), pc, rmax), self.h)
        return np.array(cov[:]), en.value, np.array(pc[:2 * rmax])

    def stats(self) -> dict:
        out = (C.c_uint64 * 5)()
        _check(lib().fskmc_stats(self.h, out), self.h)
        rr = C.c_uint64()
        _check(lib().fskmc_exact_edge_checks(self.h, C.byref(rr)), self.h)
        return dict(events=out[0], windows=out[1], ambiguous=out[2], timeouts=out[3],
                    check_failures=out[4], exact_edge_checks=rr.value)

    def workload(self, replica: int = 0) -> np.ndarray:
        info = self.info()
        lx, ly = self.sizes[replica]
        out = np.zeros((lx // info["qx"]) * (ly // info["qy"]), np.int32)
        _check(lib().fskmc_workload(self.h, replica, out.ctypes.data_as(C.POINTER(C.c_int32))),
               self.h)
        return out

    def sync(self):
        _check(lib().fskmc_sync(self.h), self.h)


def schedule(scheme, dt: float, T: float, seed: int = 0, replica: int = 0, w0: int = 0):
    """fskmc_schedule: (colours, lengths) of the windows of a run."""
    s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    n = C.c_int64()
    _check(lib().fskmc_schedule(s, dt, T, seed, replica, w0, None, None, 0, C.byref(n)))
    col = np.zeros(max(n.value, 1), np.int32)
    h = np.zeros(max(n.value, 1), np.float64)
    _check(lib().fskmc_schedule(s, dt, T, seed, replica, w0, col.ctypes.data, h.ctypes.data,
                                n.value, C.byref(n)))
    return col[:n.value], h[:n.value]


def selftest_divide(a, b) -> int:
    """fskmc_selftest_divide: mismatches of the kernel's divide vs the hardware's."""
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    bad = C.c_uint32()
    _check(lib().fskmc_selftest_divide(a.ctypes.data, b.ctypes.data, len(a), C.byref(bad)))
    return bad.value


def selftest_log(n) -> np.ndarray:
    """fskmc_selftest_log: the device's -log(n 2^-53) for integers n in [1, 2^53]."""
    n = np.ascontiguousarray(n, np.uint64)
    out = np.empty(len(n), np.float64)
    _check(lib().fskmc_selftest_log(n.ctypes.data, len(n), out.ctypes.data))
    return out


def autotune(batch, model, scheme, dt, clock="FP32", engine="PERSISTENT", coverage=0.5,
             seed=0, stream=None):
    """fskmc_autotune: fastest (q, warps per block, events/s) for a batch."""
    n = len(batch)
    lats = (Lattice * n)(*[Lattice(b["lx"], b["ly"], 0) for b in batch])
    rts = (Rates * n)(*[_rates(b["rates"]) for b in batch])
    cell = CellShape()
    wpb = C.c_int32()
    rate = C.c_double()
    m = MODELS[model] if isinstance(model, str) else int(model)
    s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    st = lib().fskmc_autotune(n, lats, m, rts, s, dt, CLOCKS[clock], ENGINES[engine], coverage,
                              seed, _stream_ptr(stream), C.byref(cell), C.byref(wpb),
                              C.byref(rate))
    _check(st)
    return (cell.qx, cell.qy), wpb.value, rate.value


def observables_noalloc(lattice, lx: int, ly: int, model, rmax: int = 0, stream=None):
    """fskmc_observables_noalloc on a device lattice (a CUDA uint8 tensor or a
    raw device pointer): the observables without any allocation by the
    library. Calls that overlap on the GPU share one scratch array and race."""
    p = lattice if isinstance(lattice, int) else lattice.data_ptr()
    m = MODELS[model] if isinstance(model, str) else int(model)
    cov = (C.c_double * 3)()
    en = C.c_double()
    pc = (C.c_double * max(2 * rmax, 1))()
    st = lib().fskmc_observables_noalloc(p, lx, ly, m, _stream_ptr(stream), cov, C.byref(en), pc,
                                         rmax)
    if st != OK:
        raise FskmcError(st, "fskmc_observables_noalloc rejected the call")
    return np.array(cov[:]), en.value, np.array(pc[:2 * rmax])

"""The C-ABI library loads and exports every entry point include/fskmc.h
declares; argument validation that happens before any device work is
checked here without a GPU."""
import ctypes as C
import os
import re

import pytest

import paper_1105_4673_gb300 as F
from paper_1105_4673_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.lib()


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fskmc_[a-z_0-9]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "fskmc_create" in names and "fskmc_run" in names and "fskmc_observables" in names
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(F.EXPORTS) | {n for n in names if n.startswith("fskmc_")}
    assert set(F.EXPORTS) <= names


def _create(lib, lx, ly, model, q, rates=None):
    h = C.c_void_p()
    st = lib.fskmc_create(C.byref(F.Lattice(lx, ly, 0)), model, C.byref(F._rates(rates or {})),
                          F.CellShape(*q), None, C.byref(h))
    return st, h


@pytest.mark.parametrize("lx,ly,model,q,rates", [
    (64, 64, 0, (6, 8), {}),            # 64 not a multiple of 12
    (64, 64, 0, (0, 8), {}),            # bad cell
    (64, 64, 0, (40, 8), {}),           # q > 32
    (16, 16, 3, (1, 2), {}),            # two-site model with q < 2
    (4, 4, 2, (2, 2), {}),              # diffusion halo needs lx >= qx + 4
    (64, 64, 0, (8, 8), dict(ka=-1.0)),  # negative rate
    (64, 64, 3, (8, 8), dict(yA=1.5)),  # yA outside [0,1]
    (64, 64, 7, (8, 8), {}),            # unknown model
    (64, 64, 1, (8, 8), dict(betaJ=float("nan"))),
    (64, 2, 4, (8, 1), {}),             # ring: ly must be 1
    (64, 1, 4, (8, 2), {}),             # ring: qy must be 1
    (96, 1, 4, (64, 1), {}),            # ring of 96 not a multiple of 128
    (4096, 1, 4, (2048, 1), {}),        # ring cell longer than 1024
    (64, 1, 4, (8, 1), dict(betah=float("inf"))),
    (64, 1, 0, (8, 1), {}),             # a 2D model on one row
])
def test_create_rejects_invalid_arguments(lib, lx, ly, model, q, rates):
    st, h = _create(lib, lx, ly, model, q, rates)
    assert st == F.EINVAL and not h.value
    assert lib.fskmc_last_error(None).decode()


def test_null_context_calls_fail_cleanly(lib):
    assert lib.fskmc_run(None, 0, 0.1, 1.0, 1) == F.EINVAL
    assert lib.fskmc_sync(None) == F.EINVAL
    assert lib.fskmc_stats(None, None) == F.EINVAL
    assert lib.fskmc_exact_edge_checks(None, None) == F.EINVAL
    assert lib.fskmc_set_edge_screen(None, 1) == F.EINVAL
    lib.fskmc_destroy(None)


@pytest.mark.parametrize("scheme", ["LIE", "STRANG", "RANDOM", "RANDOM_ORDER"])
@pytest.mark.parametrize("replica,w0", [(0, 0), (5, 1234), (77, 2**31)])
def test_schedule_matches_oracle(lib, scheme, replica, w0):
    """Row a2 (schedules, Section 3): the library's window list equals the
    oracle's, window for window (host code, no GPU needed)."""
    import numpy as np
    import oracle
    col, h = F.schedule(scheme, 0.05, 3.0, seed=0xABCDEF, replica=replica, w0=w0)
    ocol, oh = oracle.schedule(scheme, 0.05, 3.0, seed=0xABCDEF, replica=replica, w0=w0)
    assert np.array_equal(col, ocol) and np.array_equal(h, oh)
    with pytest.raises(F.FskmcError):
        F.schedule(scheme, 0.07, 1.0)


@pytest.mark.parametrize("lx,ly,model,q", [(64, 64, 3, (8, 8)),    # ZGB has three states
                                           (48, 48, 1, (8, 8)),    # lx not a multiple of 32
                                           (64, 64, 2, (8, 8)),    # diffusion: not a spin flip
                                           (48, 1, 4, (8, 1))])    # ring of 48 sites
def test_bitpacked_validation(lib, lx, ly, model, q):
    h = C.c_void_p()
    st = lib.fskmc_create(C.byref(F.Lattice(lx, ly, 1)), model, C.byref(F._rates({})),
                          F.CellShape(*q), None, C.byref(h))
    assert st == F.EINVAL and not h.value


def test_sides_above_the_limit_are_refused(lib):
    """Lattice sides above FSKMC_MAX_SIDE (2^30) are refused before any
    device work, for rings too (a ring of 2^31 - 2 sites would take the
    observables' site arithmetic past 32 bits), by the context constructor
    and by the allocation-free observables."""
    big = 2 ** 31 - 2
    with pytest.raises(F.FskmcError) as e:
        F.Context(big, 1, "ISING1D", dict(ka=1.0, kd=1.0, betaJ=1.0), (1, 1))
    assert e.value.status == F.EINVAL and "side" in str(e.value)
    with pytest.raises(F.FskmcError) as e:
        F.Context(2 ** 30 + 2, 2, "ADSDES", dict(ka=1.0, kd=1.0, betaJ=1.0), (1, 1))
    assert e.value.status == F.EINVAL
    cov = (C.c_double * 3)()
    en = C.c_double()
    for lx, ly in ((big, 1), (2 ** 30 + 2, 1), (1, 2 ** 30 + 2)):
        st = lib.fskmc_observables_noalloc(16, lx, ly, F.MODELS["ISING1D"], None, cov, C.byref(en),
                                           None, 0)
        assert st == F.EINVAL, (lx, ly)

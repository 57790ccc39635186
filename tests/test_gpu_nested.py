"""The nested (two-level) scheme on the GPU, Section 5 (Eq. sublatt2, Eq.
opdecomp2): super-cells as thread blocks held in shared memory for a whole
outer window, sub-cells as warps. With the binary64 clock the lattices,
event counts and per-sub-cell workloads equal the oracle's nested run bit
for bit, across outer and inner schedules, inner step counts, ragged
sub-cells, byte and bit-packed storage and batches; the binary32 clock
follows the J = 0 closed form."""
import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from oracle import closed_forms as CF

pytestmark = pytest.mark.gpu

RATES = {"ISING": dict(ka=1.0, kd=1.0, betaJ=0.4407), "ADSDES": dict(ka=1.0, kd=1.0, betaJ=1.0)}

# (model, lx, ly, super-cell, sub-cell, packed)
GEOMS = [
    ("ISING", 128, 128, (32, 32), (8, 8), False),
    ("ADSDES", 96, 64, (48, 16), (8, 8), False),
    ("ISING", 48, 40, (12, 10), (6, 5), False),        # ragged sub-cells
    ("ISING", 256, 128, (64, 64), (16, 16), False),
    ("ISING", 128, 64, (32, 32), (8, 8), True),        # bit-packed lattice
    ("ADSDES", 64, 64, (16, 16), (4, 4), False),
    ("ISING", 64, 64, (32, 32), (16, 16), True),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


def _gpu(model, lx, ly, Q, q, packed, init, inner, n_in, clock="FP64", grouped=True):
    c = F.Context(lx, ly, model, RATES[model], q, bitpacked=packed)
    c.set_clock(clock)
    c.set_cell_grouping(grouped)
    c.set_nesting(Q, inner, n_in)
    c.set_state(init)
    return c


@pytest.mark.parametrize("model,lx,ly,Q,q,packed", GEOMS)
@pytest.mark.parametrize("scheme,inner,n_in", [("LIE", "LIE", 1), ("STRANG", "STRANG", 2),
                                               ("RANDOM", "LIE", 3), ("LIE", "STRANG", 1)])
@pytest.mark.parametrize("grouped", [True, False])  # sub-cells several per warp, or one per warp
def test_nested_bit_exact(model, lx, ly, Q, q, packed, scheme, inner, n_in, grouped):
    seed = 0x2E57 + lx + ly + n_in
    init = oracle.init_bernoulli(lx, ly, seed, 0.5)
    dt, T = 0.2, 1.0
    orc = oracle.FS2Run(lx, ly, Q, q, model, RATES[model], init).run(scheme, dt, T, seed, inner, n_in)
    with _gpu(model, lx, ly, Q, q, packed, init, inner, n_in, grouped=grouped) as c:
        assert c.info()["lanes_per_cell"] == (8 if grouped else 32)
        c.run(scheme, dt, T, seed)
        st = c.stats()
        g, wl = c.get_state(), c.workload()
    # a flagged inner window (an edge decision within 1e-12 of its end) would
    # need a replay; none occurs on these inputs, and the test says so
    assert orc.ambiguous == 0
    assert st["check_failures"] == 0
    assert np.array_equal(g, orc.lat)
    assert st["events"] == orc.events > 0
    assert st["windows"] == orc.windows
    assert np.array_equal(wl, orc.workload)


def test_nested_resume_and_window_calls():
    """Two runs of T/2 equal one run of T; fskmc_window runs one outer
    window with its inner schedule."""
    model, lx, ly, Q, q = "ISING", 128, 128, (32, 32), (8, 8)
    init = oracle.init_bernoulli(lx, ly, 5, 0.5)
    orc = oracle.FS2Run(lx, ly, Q, q, model, RATES[model], init).run("STRANG", 0.25, 1.0, 9, "LIE", 2)
    with _gpu(model, lx, ly, Q, q, False, init, "LIE", 2) as c:
        c.run("STRANG", 0.25, 0.5, 9)
        c.run("STRANG", 0.25, 0.5, 9)
        assert np.array_equal(c.get_state(), orc.lat) and c.stats()["events"] == orc.events
    # Lie over one step = outer windows (E, dt), (O, dt)
    orc = oracle.FS2Run(lx, ly, Q, q, model, RATES[model], init).run("LIE", 0.25, 0.25, 9, "STRANG", 1)
    with _gpu(model, lx, ly, Q, q, False, init, "STRANG", 1) as c:
        c.window(0, 0.25, 9)
        c.window(1, 0.25, 9)
        assert np.array_equal(c.get_state(), orc.lat) and c.stats()["events"] == orc.events


def test_nested_batch_equals_single_contexts():
    reps = [dict(lx=128, ly=64, rates=dict(ka=0.5, kd=1.0, betaJ=0.3)),
            dict(lx=64, ly=64, rates=dict(ka=2.0, kd=1.0, betaJ=0.8))]
    seed = 41
    with F.Context(model="ADSDES", q=(8, 8), batch=reps) as b:
        b.set_nesting((32, 32), "LIE", 2)
        b.init_random(seed, 0.5)
        b.run("LIE", 0.1, 1.0, seed)
        for r, rp in enumerate(reps):
            init = oracle.init_bernoulli(rp["lx"], rp["ly"], seed, 0.5, replica=r)
            orc = oracle.FS2Run(rp["lx"], rp["ly"], (32, 32), (8, 8), "ADSDES", rp["rates"], init,
                                replica=r).run("LIE", 0.1, 1.0, seed, "LIE", 2)
            assert orc.ambiguous == 0
            assert np.array_equal(b.get_state(r), orc.lat), f"replica {r}"


def test_nested_fp32_noninteracting_closed_form():
    lx = ly = 512
    ka, kd, T = 2.0, 1.0, 1.0
    with F.Context(lx, ly, "ADSDES", dict(ka=ka, kd=kd, betaJ=0.0), (16, 16)) as c:
        c.set_clock("FP32")
        c.set_nesting((64, 64), "STRANG", 2)
        c.init_random(3, 0.5)
        th0 = c.get_state().mean()
        c.run("LIE", 0.1, T, 3)
        got = c.get_state().mean()
    want = CF.coverage_noninteracting(T, th0, ka, kd)
    assert abs(got - want) < 4 * np.sqrt(want * (1 - want) / (lx * ly))


def test_nested_rejects_bad_shapes():
    with F.Context(64, 64, "ISING", RATES["ISING"], (8, 8)) as c:
        for Q in ((8, 8), (24, 16), (64, 64)):  # one sub-cell across; odd count; lattice not 2 Q
            with pytest.raises(F.FskmcError):
                c.set_nesting(Q, "LIE", 1)
        with pytest.raises(F.FskmcError):
            c.set_nesting((16, 16), "RANDOM", 1)
        with pytest.raises(F.FskmcError):
            c.set_nesting((16, 16), "LIE", 0)
    with F.Context(64, 64, "ZGB", dict(yA=0.5, kr=1.0, kd=0.1), (8, 8)) as c:
        with pytest.raises(F.FskmcError):
            c.set_nesting((16, 16), "LIE", 1)

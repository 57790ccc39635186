"""Grouped window kernels (several small spin-flip cells per warp, in
lockstep): bit-identical to one cell per warp and to the oracle, for both
engines, both clocks and both storages, with partly filled warps, cells of
every grouped width and cells whose event counts differ widely within a
warp."""
import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from gpu_util import gpu_ctx, match_oracle

pytestmark = pytest.mark.gpu

RATES = {
    "ADSDES": dict(ka=1.0, kd=1.0, betaJ=1.0),
    "ISING": dict(ka=1.0, kd=1.0, betaJ=0.4407),
    "ISING1D": dict(ka=1.0, kd=1.0, betaJ=2.0, betah=2.0),
}

# (model, lx, ly, q, lanes per cell): active cells not a multiple of the
# cells per warp in most rows
GEOMS = [
    ("ISING", 12, 12, (2, 2), 8),       # 18 active cells: 4 full warps + 2 cells
    ("ISING", 96, 48, (16, 8), 8),      # 18 active 128-site cells
    ("ISING", 96, 64, (16, 16), 8),     # the benchmark's cell shape
    ("ADSDES", 128, 64, (32, 16), 16),  # 512-site cells: 2 per warp
    ("ADSDES", 60, 40, (6, 5), 8),      # ragged cells
    ("ISING1D", 576, 1, (32, 1), 4),    # 9 active ring cells: 8 per warp + 1
    ("ISING1D", 1000, 1, (100, 1), 4),
    ("ISING1D", 2560, 1, (256, 1), 8),
    ("ISING1D", 3072, 1, (512, 1), 16),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


def _run(model, lx, ly, q, init, scheme, dt, T, seed, clock, engine, grouped, packed=False):
    c = F.Context(lx, ly, model, RATES[model], q, bitpacked=packed)
    try:
        c.set_clock(clock)
        c.set_engine(engine)
        c.set_cell_grouping(grouped)
        c.set_state(init)
        c.run(scheme, dt, T, seed)
        st = c.stats()
        return c.get_state(), st, c.workload(), c.info()
    finally:
        c.close()


@pytest.mark.parametrize("model,lx,ly,q,lanes", GEOMS)
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_grouped_matches_oracle_fp64(model, lx, ly, q, lanes, engine):
    seed = 0x6A0 + lx + ly
    init = oracle.init_bernoulli(lx, ly, seed, 0.5)
    dt, T = 0.1, 1.0
    orc = oracle.FSRun(lx, ly, *q, model, RATES[model], init).run("LIE", dt, T, seed)
    lat, st, wl, info = _run(model, lx, ly, q, init, "LIE", dt, T, seed, "FP64", engine, True)
    assert info["lanes_per_cell"] == lanes
    assert st["check_failures"] == 0 and st["timeouts"] == 0
    assert st["events"] > 0
    match_oracle((lat, st["events"], wl), orc,
                 lambda: gpu_ctx(lx, ly, q, model, RATES[model], init, engine=engine, grouped=True),
                 lambda: oracle.FSRun(lx, ly, *q, model, RATES[model], init), "LIE", dt, T, seed,
                 what=f"grouped {model} {lx}x{ly} q={q} {engine}")


@pytest.mark.parametrize("model,lx,ly,q,lanes", GEOMS)
@pytest.mark.parametrize("clock", ["FP64", "FP32"])
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_grouped_equals_one_cell_per_warp(model, lx, ly, q, lanes, clock, engine):
    seed = 0x6A1 + lx
    init = oracle.init_bernoulli(lx, ly, seed, 0.5)
    a = _run(model, lx, ly, q, init, "RANDOM_ORDER", 0.2, 2.0, seed, clock, engine, True)
    b = _run(model, lx, ly, q, init, "RANDOM_ORDER", 0.2, 2.0, seed, clock, engine, False)
    assert a[3]["lanes_per_cell"] == lanes and b[3]["lanes_per_cell"] == 32
    assert np.array_equal(a[0], b[0])
    assert a[1]["events"] == b[1]["events"] and a[1]["events"] > 0
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("clock", ["FP64", "FP32"])
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_grouped_packed_storage(clock, engine):
    """Bit-packed lattice with 16-wide and 8-wide cells (two cells of a
    warp, or a cell and its inactive neighbour, share a 32-bit word)."""
    for lx, ly, q in ((256, 128, (16, 16)), (128, 64, (8, 8))):
        seed = 0x6A2 + lx
        init = oracle.init_bernoulli(lx, ly, seed, 0.5)
        a = _run("ISING", lx, ly, q, init, "STRANG", 0.5, 3.0, seed, clock, engine, True, packed=True)
        b = _run("ISING", lx, ly, q, init, "STRANG", 0.5, 3.0, seed, clock, engine, False, packed=False)
        assert np.array_equal(a[0], b[0]) and a[1]["events"] == b[1]["events"]
        if clock == "FP64":
            orc = oracle.FSRun(lx, ly, *q, "ISING", RATES["ISING"], init).run("STRANG", 0.5, 3.0, seed)
            match_oracle((a[0], a[1]["events"], a[2]), orc,
                         lambda: gpu_ctx(lx, ly, q, "ISING", RATES["ISING"], init, engine=engine,
                                         grouped=True, packed=True),
                         lambda: oracle.FSRun(lx, ly, *q, "ISING", RATES["ISING"], init),
                         "STRANG", 0.5, 3.0, seed, what=f"packed {lx}x{ly} q={q} {engine}")


@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_grouped_uneven_cells_in_a_warp(engine):
    """A Gaussian bump of occupied sites on an empty lattice: neighbouring
    cells of one warp run very different numbers of events, so groups leave
    the lockstep loop at very different iterations."""
    lx, ly, q = 128, 128, (8, 8)
    rates = dict(ka=0.05, kd=1.0, betaJ=3.0)
    out = []
    for grouped in (True, False):
        with F.Context(lx, ly, "ADSDES", rates, q) as c:
            c.set_engine(engine)
            c.set_cell_grouping(grouped)
            c.init_bump(5, 0.95, 12.0, 1)
            init = c.get_state()
            c.run("LIE", 0.5, 4.0, 17)
            out.append((c.get_state(), c.stats()["events"], c.workload()))
    wl = out[0][2]
    assert wl.max() > 4 * max(1, np.median(wl))  # uneven indeed
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])
    orc = oracle.FSRun(lx, ly, *q, "ADSDES", rates, init).run("LIE", 0.5, 4.0, 17)
    match_oracle(out[0], orc, lambda: gpu_ctx(lx, ly, q, "ADSDES", rates, init, engine=engine, grouped=True),
                 lambda: oracle.FSRun(lx, ly, *q, "ADSDES", rates, init), "LIE", 0.5, 4.0, 17,
                 what=f"bump start {engine}")


@pytest.mark.parametrize("clock", ["FP64", "FP32"])
def test_grouped_persistent_uneven_batch(clock):
    """Replicas of different sizes and rates in one persistent launch: a
    task's cells may straddle two replicas."""
    reps = [dict(lx=32, ly=32, rates=dict(ka=0.5, kd=1.0, betaJ=0.3)),
            dict(lx=64, ly=48, rates=dict(ka=2.0, kd=1.0, betaJ=0.8)),
            dict(lx=48, ly=16, rates=dict(ka=1.0, kd=1.0, betaJ=0.0)),
            dict(lx=16, ly=16, rates=dict(ka=0.1, kd=1.0, betaJ=0.5))]
    seed = 77
    res = []
    for grouped in (True, False):
        with F.Context(model="ADSDES", q=(8, 8), batch=reps) as b:
            b.set_engine("PERSISTENT")
            b.set_clock(clock)
            b.set_cell_grouping(grouped)
            b.init_random(seed, 0.5)
            b.run("LIE", 0.1, 2.0, seed)
            assert b.stats()["timeouts"] == 0
            res.append(([b.get_state(r) for r in range(len(reps))], b.stats()["events"]))
    for r in range(len(reps)):
        assert np.array_equal(res[0][0][r], res[1][0][r]), f"replica {r}"
    assert res[0][1] == res[1][1]


def test_grouping_switch_rejects_bad_values():
    with F.Context(64, 64, "ISING", RATES["ISING"], (8, 8)) as c:
        with pytest.raises(F.FskmcError):
            F._check(F.lib().fskmc_set_cell_grouping(c.h, 3), c.h)
        with pytest.raises(F.FskmcError):
            F._check(F.lib().fskmc_set_edge_screen(c.h, 2), c.h)
        assert c.info()["lanes_per_cell"] == 8  # auto: plain engine
        c.set_cell_grouping(False)
        assert c.info()["lanes_per_cell"] == 32
        c.set_cell_grouping(True)
        c.set_engine("PERSISTENT")
        assert c.info()["lanes_per_cell"] == 8
        c.set_cell_grouping("AUTO")
        assert c.info()["lanes_per_cell"] == 8
        c.set_clock("FP32")
        assert c.info()["lanes_per_cell"] == 8
    with F.Context(64, 64, "ZGB", dict(yA=0.5, kr=1.0, kd=0.0), (8, 8)) as c:
        assert c.info()["lanes_per_cell"] == 32  # two-site models take a whole warp
    with F.Context(64, 24, "ZGB", dict(yA=0.5, kr=1.0, kd=0.0), (32, 6)) as c:
        c.set_clock("FP32")
        assert c.info()["lanes_per_cell"] == 16  # rows not a multiple of 4: two cells per warp
    with F.Context(64, 64, "ZGB", dict(yA=0.5, kr=1.0, kd=0.0), (32, 32)) as c:
        assert c.info()["lanes_per_cell"] == 32  # binary64 clock: one cell per warp
        c.set_clock("FP32")
        assert c.info()["lanes_per_cell"] == 4  # eight 32-wide cells per warp
        c.set_cell_grouping(False)
        assert c.info()["lanes_per_cell"] == 32


# High rates (about 10^4 events per cell-window), so that a few percent of
# the cell-windows end within the screened edge check's error bound and take
# that decision from the binary64 clock; and a window too long for the
# screen (every decision in binary64). The two-site models run one cell per
# warp.
SCREEN_CASES = [
    ("ADSDES", 1024, 512, (32, 16), dict(ka=40.0, kd=40.0, betaJ=0.5), 1.0),
    ("ISING", 1024, 512, (16, 16), dict(ka=40.0, kd=40.0, betaJ=0.3), 1.0),
    ("ISING1D", 65536, 1, (128, 1), dict(ka=40.0, kd=40.0, betaJ=1.0, betah=0.5), 1.0),
    ("ADSDES", 256, 128, (8, 8), dict(ka=1e-16, kd=1e-16, betaJ=0.5), 2e15),
    ("ZGB", 512, 512, (32, 32), dict(yA=0.5, kr=50.0, kd=5.0), 4.0),
    ("DIFFUSION", 512, 512, (32, 32), dict(ka=4.0, kd=4.0, betaJ=0.5, nu=20.0), 1.0),
]


@pytest.mark.parametrize("model,lx,ly,q,rates,dt", SCREEN_CASES)
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_screened_edge_check_matches_binary64(model, lx, ly, q, rates, dt, engine):
    """Binary64 window-edge decisions screened by a bounded binary32
    estimate, with the binary64 clock deciding the events inside the bound:
    lattices, events, workloads and ambiguity counts equal those of every
    decision taken from the binary64 divide, in the grouped and the one-cell
    kernels."""
    seed = 0x5C + lx
    init = oracle.init_bernoulli(lx, ly, seed, 0.5)
    if model == "ZGB":
        init = np.zeros_like(init)  # an empty surface
    spin = model in ("ADSDES", "ISING", "ISING1D")
    forms = [(g, sc) for g in ((True, False) if spin else (False,)) for sc in (True, False)]
    res = {}
    for grouped, screen in forms:
        with F.Context(lx, ly, model, rates, q) as c:
            c.set_engine(engine)
            c.set_cell_grouping(grouped)
            c.set_edge_screen(screen)
            c.set_state(init)
            c.run("LIE", dt, 4.0 * dt, seed)
            res[grouped, screen] = (c.get_state(), c.stats(), c.workload(), c.info()["lanes_per_cell"])
    lr, sr, wr, _ = res[False, False]
    assert sr["events"] > 0 and sr["exact_edge_checks"] >= sr["events"]  # every decision in binary64
    for (grouped, screen), (la, sa, wa, lanes) in res.items():
        assert (lanes < 32) == grouped
        assert sa["check_failures"] == 0 and sa["timeouts"] == 0
        assert sa["events"] == sr["events"] and sa["ambiguous"] == sr["ambiguous"], (grouped, screen)
        assert np.array_equal(la, lr), (grouped, screen)
        assert np.array_equal(wa, wr), (grouped, screen)
        if not screen or dt > 1e15 or (engine == "PERSISTENT" and not grouped):
            # screen off, beyond its range, or the persistent one-cell kernel
            # (never screened): every decision in binary64
            assert sa["exact_edge_checks"] >= sa["events"]
        else:
            assert 0 < sa["exact_edge_checks"] < sa["events"] // 1000, (grouped, sa["exact_edge_checks"])


@pytest.mark.parametrize("model,rates", [
    ("ADSDES", dict(ka=0.75, kd=0.5, betaJ=0.0)),      # every class rate dyadic
    ("ADSDES", dict(ka=0.0, kd=3.0, betaJ=0.25)),      # a zero rate, then one dyadic class
    ("ISING", dict(ka=1.0, kd=1.0, betaJ=0.4407)),     # five unit rates, then binary64
    ("ISING", dict(ka=1.5, kd=2.0 ** -30, betaJ=0.0)),  # dyadic rates far apart
])
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_dyadic_and_zero_rates_match_oracle(model, rates, engine):
    """Dyadic rates (every fused multiply-add of the class sums exact, or
    only the leading ones), a zero rate and rates far apart: the grouped
    binary64 kernels give the same lattices and events as the oracle and
    the one-cell kernels."""
    lx, ly, q = 96, 64, (16, 16)
    seed = 0x7E5
    init = oracle.init_bernoulli(lx, ly, seed, 0.5)
    res = []
    for grouped in (True, False):
        with F.Context(lx, ly, model, rates, q) as c:
            c.set_engine(engine)
            c.set_cell_grouping(grouped)
            c.set_state(init)
            c.run("STRANG", 0.5, 3.0, seed)
            res.append((c.get_state(), c.stats()["events"], c.workload()))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] > 0
    orc = oracle.FSRun(lx, ly, *q, model, rates, init).run("STRANG", 0.5, 3.0, seed)
    match_oracle(res[0], orc, lambda: gpu_ctx(lx, ly, q, model, rates, init, engine=engine, grouped=True),
                 lambda: oracle.FSRun(lx, ly, *q, model, rates, init), "STRANG", 0.5, 3.0, seed,
                 what=f"{model} {rates} {engine}")

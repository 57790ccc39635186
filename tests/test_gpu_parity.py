"""Parity of the CUDA path with the oracle: bit-identical lattices, event
counts and workloads under the same seeds (binary64 clocks), across models,
schedules, cell shapes (including ragged cells that leave lanes idle) and
launch shapes."""
import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from gpu_util import gpu_ctx, match_oracle
from workloads import WORKLOADS, random_lattice

pytestmark = pytest.mark.gpu

RATES = {
    "ADSDES": dict(ka=1.0, kd=1.0, betaJ=1.0),
    "ISING": dict(ka=1.0, kd=1.0, betaJ=0.4407),
    "DIFFUSION": dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0),
    "ZGB": dict(yA=0.52, kr=100.0, kd=0.01),
}

# (model, lx, ly, q): several tiles, non-power-of-two and ragged cells
GEOMS = [
    ("ADSDES", 64, 64, (8, 8)),
    ("ADSDES", 4, 4, (2, 2)),
    ("ISING", 60, 40, (6, 5)),
    ("ISING", 48, 40, (12, 10)),
    ("ISING", 128, 64, (32, 32)),
    ("DIFFUSION", 48, 48, (8, 8)),
    ("DIFFUSION", 16, 24, (4, 6)),
    ("DIFFUSION", 64, 64, (32, 32)),
    ("DIFFUSION", 128, 96, (32, 16)),
    ("ZGB", 64, 64, (8, 8)),
    ("ZGB", 8, 8, (2, 2)),
    ("ZGB", 96, 64, (16, 32)),
    ("ZGB", 128, 64, (32, 32)),
    ("ZGB", 64, 96, (32, 16)),
]


def _init(model, lx, ly, seed):
    if model == "ZGB":
        return random_lattice(lx, ly, 3, seed, p=[0.6, 0.2, 0.2])
    return oracle.init_bernoulli(lx, ly, seed, 0.3 if model == "DIFFUSION" else 0.5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


@pytest.mark.parametrize("model,lx,ly,q", GEOMS)
@pytest.mark.parametrize("scheme", ["LIE", "STRANG", "RANDOM", "RANDOM_ORDER"])
def test_run_bit_exact(model, lx, ly, q, scheme):
    dt = 0.05 if model != "ZGB" else 0.02
    T = 1.0 if lx * ly <= 64 * 64 else 0.5
    seed = 0xC0FFEE + lx + 7 * ly
    init = _init(model, lx, ly, seed)
    orc = oracle.FSRun(lx, ly, *q, model, RATES[model], init).run(scheme, dt, T, seed)
    with gpu_ctx(lx, ly, q, model, RATES[model], init) as c:
        c.run(scheme, dt, T, seed)
        g = c.get_state()
        st = c.stats()
        wl = c.workload()
    match_oracle((g, st["events"], wl), orc,
                 lambda: gpu_ctx(lx, ly, q, model, RATES[model], init),
                 lambda: oracle.FSRun(lx, ly, *q, model, RATES[model], init),
                 scheme, dt, T, seed, what=f"{model} {lx}x{ly} q={q} {scheme}")
    assert st["windows"] == orc.windows and st["events"] > 0


def test_workload_adsdes64_both_couplings():
    """The 64x64 adsorption/desorption workload in full (Lie, dt = 0.1,
    T = 10, 8x8 cells) at betaJ = 0 and 1."""
    w = WORKLOADS["adsdes64"]
    for bJ in (0.0, 1.0):
        rates = dict(w["rates"], betaJ=bJ)
        init = oracle.init_bernoulli(w["lx"], w["ly"], w["seed"], w["coverage"])
        orc = oracle.FSRun(w["lx"], w["ly"], *w["q"], w["model"], rates, init)
        orc.run(w["scheme"], w["dt"], w["T"], w["seed"])
        with F.Context(w["lx"], w["ly"], w["model"], rates, w["q"]) as c:
            c.init_random(w["seed"], w["coverage"])
            assert np.array_equal(c.get_state(), init)
            c.run(w["scheme"], w["dt"], w["T"], w["seed"])
            assert np.array_equal(c.get_state(), orc.lat)
            assert c.stats()["events"] == orc.events
            cov, en, pc = c.observables(0, 8)
            ocov, oen, opc = oracle.observables(w["lx"], w["ly"], w["model"], orc.lat, 8)
            assert np.array_equal(cov, ocov) and en == oen and np.array_equal(pc, opc)


@pytest.mark.parametrize("model", ["ISING", "ZGB", "DIFFUSION"])
def test_observables_bit_exact(model):
    lx, ly = 96, 80
    lat = _init(model, lx, ly, 5)
    with F.Context(lx, ly, model, RATES[model], (8, 8)) as c:
        c.set_state(lat)
        for rmax in (0, 1, 16):
            cov, en, pc = c.observables(0, rmax)
            ocov, oen, opc = oracle.observables(lx, ly, model, lat, rmax)
            assert np.array_equal(cov, ocov)
            assert (np.isnan(en) and np.isnan(oen)) or en == oen
            assert np.array_equal(pc, opc)


def test_init_matches_oracle():
    with F.Context(96, 64, "ZGB", RATES["ZGB"], (8, 8)) as c:
        c.init_random(123, 0.37)
        assert np.array_equal(c.get_state(), oracle.init_bernoulli(96, 64, 123, 0.37))
        c.init_bump(77, 0.9, 96 / 8, 1)
        assert np.array_equal(c.get_state(), oracle.init_bump(96, 64, 77, 0.9, 96 / 8, 1))


@pytest.mark.parametrize("wpb", [1, 3, 8, 16])
def test_launch_shape_invariance(wpb):
    model, lx, ly, q = "ISING", 64, 64, (8, 8)
    init = _init(model, lx, ly, 9)
    orc = oracle.FSRun(lx, ly, *q, model, RATES[model], init).run("STRANG", 0.1, 1.0, 4)
    with gpu_ctx(lx, ly, q, model, RATES[model], init, wpb=wpb) as c:
        c.run("STRANG", 0.1, 1.0, 4)
        got = (c.get_state(), c.stats()["events"], c.workload())
    match_oracle(got, orc, lambda: gpu_ctx(lx, ly, q, model, RATES[model], init, wpb=wpb),
                 lambda: oracle.FSRun(lx, ly, *q, model, RATES[model], init), "STRANG", 0.1, 1.0, 4,
                 what=f"{wpb} warps per block")


@pytest.mark.parametrize("model", ["ADSDES", "DIFFUSION", "ZGB"])
def test_resume_is_bit_exact(model):
    lx, ly, q = 64, 64, (8, 8)
    init = _init(model, lx, ly, 11)
    with gpu_ctx(lx, ly, q, model, RATES[model], init) as a, \
            gpu_ctx(lx, ly, q, model, RATES[model], init) as b:
        a.run("RANDOM", 0.05, 1.0, 3)
        b.run("RANDOM", 0.05, 0.5, 3)
        w = b.window_index
        snap = b.get_state()
        with gpu_ctx(lx, ly, q, model, RATES[model], snap) as b2:
            b2.window_index = w
            b2.run("RANDOM", 0.05, 0.5, 3)
            assert np.array_equal(a.get_state(), b2.get_state())


def test_invalid_state_rejected():
    with F.Context(16, 16, "ADSDES", RATES["ADSDES"], (4, 4)) as c:
        bad = np.zeros(256, np.uint8)
        bad[3] = 2
        with pytest.raises(F.FskmcError) as e:
            c.set_state(bad)
        assert e.value.status == F.EINVAL
        with pytest.raises(F.FskmcError):
            c.run("LIE", 0.3, 1.0, 1)  # T/dt not an integer


def test_flagged_window_takes_the_replay_path():
    """A window whose length equals cell 0's first waiting time puts that
    edge decision exactly on the window end: the oracle flags the
    cell-window, and the comparison replays the run window by window
    (resyncing at most at the flagged window) instead of skipping it."""
    import math
    lx, ly, q = 16, 16, (4, 4)
    rates = dict(ka=1.0, kd=1.0, betaJ=0.0)  # every site rate 1: lambda = 16 in every cell
    seed = 0x5151
    o = oracle.philox([0, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])  # (e, w, m, replica|tag 0)
    u = ((int(o[0]) << 21 | int(o[1]) >> 11) + 1) * 2.0 ** -53
    h = -math.log(u) / 16.0
    init = oracle.init_bernoulli(lx, ly, seed, 0.5)
    orc = oracle.FSRun(lx, ly, *q, "ADSDES", rates, init).run("LIE", h, h, seed)
    assert orc.ambiguous >= 1
    for engine in ("PLAIN", "PERSISTENT"):
        with gpu_ctx(lx, ly, q, "ADSDES", rates, init, engine=engine) as c:
            c.run("LIE", h, h, seed)
            got = (c.get_state(), c.stats()["events"], c.workload())
        n = match_oracle(got, orc, lambda: gpu_ctx(lx, ly, q, "ADSDES", rates, init, engine=engine),
                         lambda: oracle.FSRun(lx, ly, *q, "ADSDES", rates, init), "LIE", h, h, seed,
                         what=f"flagged window, {engine}")
        assert n <= 1


@pytest.mark.parametrize("model,lx,ly,packed", [
    ("ZGB", 32, 2, False), ("ZGB", 64, 8, False), ("ZGB", 1056, 40, False), ("ISING", 2048, 64, True),
    ("ADSDES", 96, 34, False), ("ISING1D", 2048, 1, False), ("ISING1D", 4096, 1, True),
    ("ZGB", 1024, 1024, False),
])
@pytest.mark.parametrize("rmax", [0, 1, 7, 32])
def test_observables_word_path_bit_exact(model, lx, ly, packed, rmax):
    """The word-parallel observables (rows of whole 32-site words, r <= 32):
    partial word chunks, lattices shorter than the staged rows, rings, both
    storages, against the oracle's site-by-site sums."""
    if rmax > lx or (ly > 1 and rmax > ly):
        pytest.skip("r beyond the lattice")
    nstates = 3 if model == "ZGB" else 2
    lat = random_lattice(lx, ly, nstates, lx + ly + rmax)
    q = (1, 1) if model != "ZGB" else (2, 2) if ly >= 4 else (2, 1)
    if model == "ZGB" and ly < 4:
        model_ctx = "ADSDES"  # a two-row lattice is too short for two-site cells; same sums
        lat = random_lattice(lx, ly, 2, lx + ly + rmax)
    else:
        model_ctx = model
    with F.Context(lx, ly, model_ctx, RATES.get(model_ctx, dict(ka=1.0, kd=1.0, betaJ=0.5)), q,
                   bitpacked=packed) as c:
        c.set_state(lat)
        cov, en, pc = c.observables(0, rmax)
    ocov, oen, opc = oracle.observables(lx, ly, model_ctx, lat, rmax)
    assert np.array_equal(cov, ocov)
    assert (np.isnan(en) and np.isnan(oen)) or en == oen
    assert np.array_equal(pc, opc)

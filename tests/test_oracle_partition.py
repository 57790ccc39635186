"""Pin the cell decomposition: every event of the generator belongs to exactly
one (colour, cell) pair (Eq. gendecomp / Eq. opdecomp), same-colour cells have
disjoint write sets, and the result of a window does not depend on the order
in which cells are processed (Eq. exact)."""
import itertools

import numpy as np
import pytest

import oracle

MODELS = ["ADSDES", "ISING", "DIFFUSION", "ZGB"]
RATES = dict(ka=1.0, kd=1.0, betaJ=0.5, nu=2.0, yA=0.5, kr=2.0)


def _all_events(lx, ly, model):
    ev = {("site", i, i) for i in range(lx * ly)}
    if model in ("DIFFUSION", "ZGB"):
        for y, x in itertools.product(range(ly), range(lx)):
            for dx, dy in [(0, -1), (1, 0), (0, 1), (-1, 0)]:
                ev.add(("slot", y * lx + x, ((y + dy) % ly) * lx + (x + dx) % lx))
    return ev


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("lx,ly,qx,qy", [(8, 8, 2, 2), (12, 8, 3, 4), (16, 16, 4, 4)])
def test_events_partitioned(model, lx, ly, qx, qy):
    lat = np.zeros(lx * ly, np.uint8)
    ncx, ncy = lx // qx, ly // qy
    seen = []
    for m in range(ncx * ncy):
        col = ((m % ncx) + (m // ncx)) % 2
        o, t, k, _ = oracle.cell_members(lx, ly, qx, qy, model, RATES, lat, m, col)
        seen += [("site" if kk == 0 else "slot", int(a), int(b)) for a, b, kk in zip(o, t, k)]
    assert len(seen) == len(set(seen)), "an event is owned twice"
    assert set(seen) == _all_events(lx, ly, model)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("lx,ly,qx,qy", [(8, 8, 2, 2), (12, 8, 3, 4), (4, 4, 2, 2)])
def test_write_sets_disjoint(model, lx, ly, qx, qy):
    ncx, ncy = lx // qx, ly // qy
    for col in (0, 1):
        cells = [m for m in range(ncx * ncy) if ((m % ncx) + (m // ncx)) % 2 == col]
        sets = [set(oracle.cell_writeset(lx, ly, qx, qy, model, m, col).tolist()) for m in cells]
        for a, b in itertools.combinations(sets, 2):
            assert not (a & b)
        if model in ("ADSDES", "ISING"):
            assert sum(len(s) for s in sets) == lx * ly // 2


@pytest.mark.parametrize("model", MODELS)
def test_cell_order_independent_and_resumable(model):
    lx = ly = 32
    init = oracle.init_bernoulli(lx, ly, 4, 0.4)
    rates = dict(ka=1.0, kd=1.0, betaJ=1.0, nu=5.0, yA=0.52, kr=10.0)
    a = oracle.FSRun(lx, ly, 4, 4, model, rates, init).run("STRANG", 0.1, 1.0, 42, order=0)
    b = oracle.FSRun(lx, ly, 4, 4, model, rates, init).run("STRANG", 0.1, 1.0, 42, order=1)
    assert np.array_equal(a.lat, b.lat) and a.events == b.events
    # resume: two half runs continue the window counter and give the same state
    c = oracle.FSRun(lx, ly, 4, 4, model, rates, init)
    c.run("STRANG", 0.1, 0.5, 42).run("STRANG", 0.1, 0.5, 42)
    assert np.array_equal(a.lat, c.lat) and a.events == c.events
    assert a.ambiguous == 0


def test_diffusion_conserves_particles():
    lx = ly = 32
    init = oracle.init_bernoulli(lx, ly, 5, 0.3)
    run = oracle.FSRun(lx, ly, 8, 8, "DIFFUSION", dict(ka=0.0, kd=0.0, betaJ=1.0, nu=10.0), init)
    run.run("RANDOM", 0.05, 1.0, 6)
    assert run.events > 1000
    assert int(run.lat.sum()) == int(init.sum())
    assert not np.array_equal(run.lat, init)


def test_zgb_species_bookkeeping():
    """Each ZGB event changes (nA, nB) by one of (+1,0), (0,+2), (-1,-1),
    (-1,0); over a run the net change must be a non-negative combination."""
    lx = ly = 16
    run = oracle.FSRun(lx, ly, 4, 4, "ZGB", dict(yA=0.52, kr=100.0, kd=0.01))
    nA = nB = 0
    for _ in range(20):
        before = np.bincount(run.lat, minlength=3)
        run.run("STRANG", 0.02, 0.02, 9)
        after = np.bincount(run.lat, minlength=3)
        dA, dB = int(after[1] - before[1]), int(after[2] - before[2])
        assert dB % 1 == 0
        nA, nB = nA + dA, nB + dB
    counts = np.bincount(run.lat, minlength=3)
    assert counts.sum() == lx * ly and counts[1] == nA and counts[2] == nB


def test_schedules():
    col, h = oracle.schedule("LIE", 0.1, 0.3)
    assert col.tolist() == [0, 1] * 3 and np.allclose(h, 0.1)
    col, h = oracle.schedule("STRANG", 0.2, 0.4)
    assert col.tolist() == [0, 1, 0] * 2 and np.allclose(h, [0.1, 0.2, 0.1] * 2)
    col, h = oracle.schedule("RANDOM", 0.1, 50.0, seed=3)
    assert len(col) == 1000 and abs(col.mean() - 0.5) < 0.07 and np.allclose(h, 0.1)
    col, h = oracle.schedule("RANDOM_ORDER", 0.1, 50.0, seed=3)
    assert len(col) == 1000 and (col[0::2] + col[1::2] == 1).all()
    with pytest.raises(ValueError):
        oracle.schedule("LIE", 0.3, 1.0)

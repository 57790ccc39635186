"""The register-resident binary32 windows of 32-wide ZGB cells (the batched
form of the 16384^2 benchmark) -- one cell per warp, two cells per warp at
two rows per lane, four at four rows per lane or eight at eight -- against
the binary64 form, which is the oracle's
arithmetic bit for bit: pair events on undirected bonds at twice the
directed rate are the same process, so over many replicas from the same
snapshot the event counts and every observable agree within 4 standard
errors -- both engines, E and O windows, cross bonds at the lattice's
periodic edges; the two engines give identical lattices, and so do the
one-cell and two-cell windows (same draws, same member numbering)."""
import numpy as np
import pytest

import paper_1105_4673_gb300 as F
from workloads import random_lattice

pytestmark = pytest.mark.gpu

RATES = dict(yA=0.52, kr=100.0, kd=0.01)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


def _runs(clock, engine, n, lx, ly, qy, scheme, dt, T, snap, grouped=True):
    reps = [dict(lx=lx, ly=ly, rates=RATES)] * n
    with F.Context(model="ZGB", q=(32, qy), batch=reps) as b:
        b.set_clock(clock)
        b.set_engine(engine)
        b.set_cell_grouping(grouped)
        for r in range(n):
            b.set_state(snap, r)
        b.run(scheme, dt, T, 0x2B32)
        st = b.stats()
        assert st["check_failures"] == 0 and st["timeouts"] == 0
        obs = []
        for r in range(n):
            cov, _, pc = b.observables(r, 2)
            obs.append(np.concatenate([cov, pc]))
        return st["events"], np.array(obs)


@pytest.mark.parametrize("lx,ly,qy,scheme,dt,T,grouped", [
    (64, 64, 32, "STRANG", 0.02, 0.1, True),
    (128, 64, 16, "LIE", 0.05, 0.2, True),
    (64, 128, 32, "RANDOM", 0.02, 0.2, True),
    (64, 64, 32, "STRANG", 0.02, 0.1, False),   # one cell per warp
    (64, 40, 5, "LIE", 0.05, 0.2, True),        # odd rows: one cell per warp
])
def test_zgb32_binary32_matches_binary64_statistically(lx, ly, qy, scheme, dt, T, grouped):
    n = 1024
    snap = random_lattice(lx, ly, 3, lx + qy, p=[0.5, 0.25, 0.25])
    ev32, o32 = _runs("FP32", "PERSISTENT", n, lx, ly, qy, scheme, dt, T, snap, grouped)
    ev64, o64 = _runs("FP64", "PLAIN", n, lx, ly, qy, scheme, dt, T, snap)
    # event counts: the totals of n independent replicas (Poisson-like: SE ~ sqrt)
    assert abs(ev32 - ev64) < 5 * np.sqrt(ev32 + ev64), (ev32, ev64)
    se = np.sqrt(o32.var(axis=0, ddof=1) / n + o64.var(axis=0, ddof=1) / n) + 1e-12
    z = np.abs(o32.mean(axis=0) - o64.mean(axis=0)) / se
    assert np.all(z < 4), z


@pytest.mark.parametrize("lx,ly,qy,scheme", [
    (128, 128, 32, "STRANG"), (256, 64, 16, "RANDOM"), (64, 96, 6, "LIE"), (128, 48, 4, "STRANG"),
    (64, 64, 2, "LIE"), (192, 64, 8, "STRANG"), (128, 96, 12, "RANDOM"),
])
def test_zgb32_engines_and_windows_agree_bitwise(lx, ly, qy, scheme):
    """Plain and persistent engines, one cell per warp and several (eight for
    rows a multiple of 8 from 16, four for a multiple of 4 from 8, else two
    for an even number of rows): the same lattice, event count and per-cell
    workloads in all four."""
    snap = random_lattice(lx, ly, 3, 7 + qy, p=[0.6, 0.2, 0.2])
    out = []
    for engine in ("PLAIN", "PERSISTENT"):
        for grouped in (True, False):
            with F.Context(lx, ly, "ZGB", RATES, (32, qy)) as c:
                c.set_clock("FP32")
                c.set_engine(engine)
                c.set_cell_grouping(grouped)
                oct8 = grouped and qy % 8 == 0 and qy >= 16
                quad = grouped and qy % 4 == 0 and qy >= 8
                pair = grouped and qy % 2 == 0 and qy >= 4
                want = 4 if oct8 else (8 if quad else (16 if pair else 32))
                assert c.info()["lanes_per_cell"] == want
                c.set_state(snap)
                c.run(scheme, 0.02, 0.4, 5)
                st = c.stats()
                assert st["check_failures"] == 0
                out.append((c.get_state(), st["events"], c.workload()))
    for g, ev, wl in out[1:]:
        assert np.array_equal(g, out[0][0]) and ev == out[0][1] > 0 and np.array_equal(wl, out[0][2])


@pytest.mark.parametrize("qy", [16, 8])  # eight and four cells per warp (persistent engine)
def test_zgb32_several_cells_per_warp_batch_equals_one_cell(qy):
    """A batch of replicas of different sizes and rates in the persistent
    engine: several cells per warp equal one cell per warp, replica by
    replica."""
    reps = [dict(lx=64, ly=64, rates=RATES), dict(lx=128, ly=64, rates=dict(yA=0.45, kr=20.0, kd=0.1)),
            dict(lx=64, ly=128, rates=dict(yA=0.6, kr=5.0, kd=0.0))]
    res = []
    for grouped in (True, False):
        with F.Context(model="ZGB", q=(32, qy), batch=reps) as b:
            b.set_clock("FP32")
            b.set_engine("PERSISTENT")
            b.set_cell_grouping(grouped)
            b.init_random(11, 0.5)
            b.run("RANDOM", 0.05, 0.5, 11)
            res.append(([b.get_state(r) for r in range(len(reps))], b.stats()["events"]))
    assert res[0][1] == res[1][1] > 0
    for r in range(len(reps)):
        assert np.array_equal(res[0][0][r], res[1][0][r]), f"replica {r}"


@pytest.mark.parametrize("colour", [0, 1])
@pytest.mark.parametrize("qy", [2, 4, 8])  # one, two and four cells per warp
def test_zgb32_single_window_outcomes_match_binary64(colour, qy):
    """One short window (about an event per active half-lattice) from a fixed
    snapshot on a 64 x 2qy lattice (32 x qy cells; at qy = 2 every site
    borders a cell edge):
    the distribution of outcomes -- which sites changed and to what -- over
    20,000 replicas of the register-resident binary32 window and of the
    binary64 window (the oracle's arithmetic) agree by a two-sample
    chi-square, so the members, their ownership (cross bonds in E windows
    horizontally, in O windows vertically) and their rates are the same."""
    from collections import Counter

    from scipy.stats import chi2_contingency
    lx, ly, n = 64, 2 * qy, 20000
    snap = random_lattice(lx, ly, 3, 99 + colour + qy, p=[0.5, 0.25, 0.25])
    reps = [dict(lx=lx, ly=ly, rates=RATES)] * n
    counts = []
    for clock in ("FP32", "FP64"):
        with F.Context(model="ZGB", q=(32, qy), batch=reps) as b:
            b.set_clock(clock)
            for r in range(n):
                b.set_state(snap, r)
            b.window(colour, 0.0004, 0x51DE + colour)
            keys = Counter()
            for r in range(n):
                g = b.get_state(r)
                idx = np.nonzero(g != snap)[0]
                keys[tuple(idx.tolist()) + tuple(g[idx].tolist())] += 1
        counts.append(keys)
    allk = set(counts[0]) | set(counts[1])
    big = [k for k in allk if counts[0][k] + counts[1][k] >= 20]
    rest = [sum(c[k] for k in allk if k not in big) for c in counts]
    table = np.array([[c[k] for k in big] + [rest[i]] for i, c in enumerate(counts)])
    assert len(big) > 20  # many distinct single events: sites and bonds of both classes
    assert chi2_contingency(table)[1] > 1e-3

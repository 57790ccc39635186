"""The register-resident binary32 window of 32-wide adsorption/desorption +
diffusion cells (Section 2's second example; classes 5 sigma + n and hops
10 + n) against the binary64 form, which is the oracle's arithmetic bit for
bit. The two number a class's members in different orders, so they agree in
law, not bit for bit: over many replicas from the same snapshot the event
counts and every observable agree within 4 standard errors, for Lie, Strang
and random-order schedules and for several cell heights; the distribution of
single-window outcomes -- which sites changed and to what -- agrees by a
two-sample chi-square in E and in O windows, so the hops across cell edges
(owned horizontally in E windows, vertically in O windows, in both
directions) and their rates are the same; and both engines give identical
lattices."""
import numpy as np
import pytest

import paper_1105_4673_gb300 as F
from workloads import random_lattice

pytestmark = pytest.mark.gpu

RATES = dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


def _runs(clock, engine, n, lx, ly, qy, scheme, dt, T, snap):
    reps = [dict(lx=lx, ly=ly, rates=RATES)] * n
    with F.Context(model="DIFFUSION", q=(32, qy), batch=reps) as b:
        b.set_clock(clock)
        b.set_engine(engine)
        for r in range(n):
            b.set_state(snap, r)
        b.run(scheme, dt, T, 0xD1F5)
        st = b.stats()
        assert st["check_failures"] == 0 and st["timeouts"] == 0
        obs = []
        for r in range(n):
            cov, energy, pc = b.observables(r, 2)
            obs.append(np.concatenate([cov, [energy], pc]))
        return st["events"], np.array(obs)


@pytest.mark.parametrize("lx,ly,qy,scheme,dt,T,engine", [
    (64, 64, 32, "LIE", 0.05, 0.2, "PERSISTENT"),
    (128, 64, 16, "STRANG", 0.05, 0.2, "PLAIN"),
    (64, 128, 32, "RANDOM_ORDER", 0.05, 0.2, "PERSISTENT"),
    (64, 40, 5, "LIE", 0.05, 0.2, "PLAIN"),      # odd cell height, rows past the cell in the warp
    (64, 8, 2, "STRANG", 0.05, 0.2, "PERSISTENT"),  # every site borders a cell edge
])
def test_diff32_binary32_matches_binary64_statistically(lx, ly, qy, scheme, dt, T, engine):
    n = 1024
    snap = random_lattice(lx, ly, 2, lx + qy, p=[0.6, 0.4])
    ev32, o32 = _runs("FP32", engine, n, lx, ly, qy, scheme, dt, T, snap)
    ev64, o64 = _runs("FP64", "PLAIN", n, lx, ly, qy, scheme, dt, T, snap)
    # event counts: the totals of n independent replicas (Poisson-like: SE ~ sqrt)
    assert abs(ev32 - ev64) < 5 * np.sqrt(ev32 + ev64), (ev32, ev64)
    se = np.sqrt(o32.var(axis=0, ddof=1) / n + o64.var(axis=0, ddof=1) / n) + 1e-12
    z = np.abs(o32.mean(axis=0) - o64.mean(axis=0)) / se
    assert np.all(z < 4), z


@pytest.mark.parametrize("lx,ly,qy,scheme", [(128, 128, 32, "RANDOM_ORDER"), (64, 96, 6, "LIE")])
def test_diff32_engines_agree_bitwise(lx, ly, qy, scheme):
    snap = random_lattice(lx, ly, 2, 7 + qy, p=[0.7, 0.3])
    out = []
    for engine in ("PLAIN", "PERSISTENT"):
        with F.Context(lx, ly, "DIFFUSION", RATES, (32, qy)) as c:
            c.set_clock("FP32")
            c.set_engine(engine)
            c.set_state(snap)
            c.run(scheme, 0.05, 0.5, 5)
            st = c.stats()
            assert st["check_failures"] == 0
            out.append((c.get_state(), st["events"], c.workload()))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1] > 0
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("colour", [0, 1])
@pytest.mark.parametrize("qy", [2, 4])
def test_diff32_single_window_outcomes_match_binary64(colour, qy):
    """One short window (about an event per active half-lattice) from a fixed
    snapshot on a 64 x 8 lattice (32 x qy cells): the distribution of
    outcomes over 20,000 replicas of the register-resident binary32 window
    and of the binary64 window agree by a two-sample chi-square."""
    from collections import Counter

    from scipy.stats import chi2_contingency
    lx, ly, n = 64, 8, 20000  # the two-site halo needs ly >= qy + 4
    snap = random_lattice(lx, ly, 2, 99 + colour + qy, p=[0.55, 0.45])
    reps = [dict(lx=lx, ly=ly, rates=RATES)] * n
    counts = []
    for clock in ("FP32", "FP64"):
        with F.Context(model="DIFFUSION", q=(32, qy), batch=reps) as b:
            b.set_clock(clock)
            for r in range(n):
                b.set_state(snap, r)
            b.window(colour, 0.0012, 0x51DE + colour)
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
    assert len(big) > 20  # many distinct single events: adsorptions, desorptions and hops
    assert chi2_contingency(table)[1] > 1e-3

"""Pin the oracle's rate classes to the paper's per-site rate formulas.

The brute-force module writes each model's rates per site, straight from
Eq. adsdesrate, Eq. Arrhenius and Table COrates. The oracle's total rate
(sum over rate classes, Eq. totalrate) must equal the brute-force exit rate
-Q[s, s] on every configuration of small lattices, and the Ising Arrhenius
rates must satisfy detailed balance with the Gibbs measure of Section 7."""
import numpy as np
import pytest

import oracle
import oracle.brute as B

CASES = [
    ("ADSDES", dict(ka=0.7, kd=1.3, betaJ=1.0)),
    ("ISING", dict(ka=1.0, kd=1.0, betaJ=0.4407)),
    ("DIFFUSION", dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0)),
    ("ZGB", dict(yA=0.52, kr=100.0, kd=0.01)),
]


@pytest.mark.parametrize("model,rates", CASES)
def test_total_rate_matches_paper_formulas(model, rates):
    lx, ly = (3, 3) if model != "ZGB" else (3, 2)
    Q = B.generator(lx, ly, model, rates)
    base = 3 if model == "ZGB" else 2
    S = B.decode(lx, ly, base)
    exit_rate = -Q.diagonal()
    rng = np.random.default_rng(1)
    for code in rng.choice(len(S), size=min(200, len(S)), replace=False):
        lam, _ = oracle.total_rate(lx, ly, model, rates, S[code].astype(np.uint8))
        assert lam == pytest.approx(exit_rate[code], rel=1e-12, abs=1e-12)


def test_zgb_counts_per_class():
    # a hand-checkable 4x1-periodic row embedded in a 4x4 lattice
    lat = np.zeros((4, 4), np.uint8)
    lat[0, :] = [1, 2, 0, 0]
    lam, n = oracle.total_rate(4, 4, "ZGB", dict(yA=0.5, kr=4.0, kd=0.25), lat)
    empty = 14
    # directed empty-empty slots: every empty site, each empty neighbour
    ee = sum(1 for y in range(4) for x in range(4) for dx, dy in B.DIRS
             if lat[y, x] == 0 and lat[(y + dy) % 4, (x + dx) % 4] == 0)
    assert n.tolist() == [empty, ee, 2, 1]
    assert lam == pytest.approx(0.5 * empty + 0.125 * ee + 1.0 * 2 + 0.25)


@pytest.mark.parametrize("betaJ", [0.2, 0.4407, 0.6])
def test_ising_detailed_balance(betaJ):
    Q = B.generator(3, 3, "ISING", dict(ka=1.0, kd=1.0, betaJ=betaJ))
    pi = B.gibbs_ising(3, 3, betaJ)
    assert np.abs(Q.T @ pi).max() < 1e-12 * np.abs(Q.diagonal()).max()
    # and the oracle's class rates obey the same ratio: r(0,n)/r(1,n) =
    # exp(-beta dH) with dH = -K n + h for adding a particle, K = 4J, h = 2K
    r = oracle.rates("ISING", ka=1.0, kd=1.0, betaJ=betaJ)
    for n in range(5):
        assert r[n] / r[5 + n] == pytest.approx(np.exp(4 * betaJ * n - 8 * betaJ), rel=1e-14)


def test_rates_values():
    r = oracle.rates("ADSDES", ka=2.0, kd=3.0, betaJ=0.5)
    assert np.allclose(r[:5], 2.0) and np.allclose(r[5:], 3.0 * np.exp(-0.5 * np.arange(5)))
    r = oracle.rates("DIFFUSION", ka=1.0, kd=1.0, betaJ=2.0, nu=10.0)
    assert np.allclose(r[10:], 10.0 * np.exp(-2.0 * np.arange(5)))
    r = oracle.rates("ZGB", yA=0.52, kr=100.0, kd=0.01)
    assert np.allclose(r, [0.52, 0.12, 25.0, 0.01])

"""Pin the oracle to closed forms: non-interacting adsorption/desorption and
the Onsager magnetisation (Eq. exactcov2d)."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as CF


@pytest.mark.parametrize("scheme", ["LIE", "STRANG", "RANDOM", "RANDOM_ORDER"])
def test_noninteracting_coverage_every_scheme(scheme):
    """With J = 0 the sites are independent and E and O commute, so every
    schedule is exact. Under RANDOM an E site has evolved dt times the number
    of E windows (and likewise O), which the oracle's schedule tells."""
    lx = ly = 64
    ka, kd, theta0, dt, T = 1.0, 1.0, 0.5, 0.1, 1.0
    seeds = range(8)
    cov_e, cov_o, exp_e, exp_o = [], [], [], []
    q = 8
    cx = (np.arange(lx) // q)[None, :]
    cy = (np.arange(ly) // q)[:, None]
    emask = ((cx + cy) % 2 == 0).reshape(-1)
    for s in seeds:
        init = oracle.init_bernoulli(lx, ly, 100 + s, theta0)
        run = oracle.FSRun(lx, ly, q, q, "ADSDES", dict(ka=ka, kd=kd, betaJ=0.0), init)
        run.run(scheme, dt, T, 1000 + s)
        col, h = oracle.schedule(scheme, dt, T, 1000 + s)
        tE, tO = h[col == 0].sum(), h[col == 1].sum()
        th0e, th0o = init[emask].mean(), init[~emask].mean()
        cov_e.append(run.lat[emask].mean())
        cov_o.append(run.lat[~emask].mean())
        exp_e.append(CF.coverage_noninteracting(tE, th0e, ka, kd))
        exp_o.append(CF.coverage_noninteracting(tO, th0o, ka, kd))
    n_each = emask.sum() * len(seeds)
    for got, want in ((cov_e, exp_e), (cov_o, exp_o)):
        got, want = np.mean(got), np.mean(want)
        se = np.sqrt(want * (1 - want) / n_each)
        assert abs(got - want) < 4 * se, (got, want, se)


def test_noninteracting_coverage_ssa():
    lx = ly = 32
    init = oracle.init_bernoulli(lx, ly, 3, 0.2)
    lat, _ = oracle.ssa_run(lx, ly, "ADSDES", dict(ka=2.0, kd=0.5, betaJ=0.0), init, 0.4, 9)
    want = CF.coverage_noninteracting(0.4, init.mean(), 2.0, 0.5)
    se = np.sqrt(want * (1 - want) / lat.size)
    assert abs(lat.mean() - want) < 4 * se


def _ising_time_average(betaJ, T, burn, dt, seed):
    lx = ly = 64
    run = oracle.FSRun(lx, ly, 8, 8, "ISING", dict(ka=1.0, kd=1.0, betaJ=betaJ),
                       np.ones(lx * ly, np.uint8))
    run.run("LIE", dt, burn, seed)
    ms = []
    for _ in range(int(round((T - burn) / 1.0))):
        run.run("LIE", dt, 1.0, seed)
        ms.append(2.0 * run.lat.mean() - 1.0)
    return np.array(ms)


def test_onsager_ordered_phase():
    """Below T_c the time-averaged |m| approaches Onsager's value; at
    betaJ = 0.6 the correlation length is about one site, so a 64^2 lattice
    and a Lie step of 0.1 leave a bias well below the 0.005 tolerance."""
    ms = _ising_time_average(0.6, 300.0, 50.0, 0.1, 7)
    want = CF.onsager_magnetisation(0.6)
    assert abs(np.abs(ms).mean() - want) < 0.005, (np.abs(ms).mean(), want)


def test_disordered_phase_relaxes():
    ms = _ising_time_average(0.3, 200.0, 100.0, 0.25, 8)
    assert abs(ms.mean()) < 0.05
    assert CF.onsager_magnetisation(0.3) == 0.0


def test_onsager_closed_form_values():
    # the critical point: sinh(beta_c K / 2) = 1 with K = 4J
    assert np.sinh(2 * CF.BETA_C_J) == pytest.approx(1.0)
    assert CF.onsager_magnetisation(0.6) == pytest.approx(0.97362, abs=2e-5)

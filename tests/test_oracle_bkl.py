"""Pin the oracle's class-list (BKL) serial SSA: the same process as the
direct-recount SSA (the serial Gillespie algorithm, Eqs. totalrate and
skeleton), so the law of its final states must equal e^{TQ} on tiny
lattices (chi-square, with a power check), and its observables must equal
the direct form's over replicas on a larger lattice."""
import numpy as np
import pytest

import oracle
import oracle.brute as B
from stats_util import chisq_pvalue

M = 20000
P_OK = 1e-3


def _bkl_ensemble(lx, ly, model, rates, init, T, seed, n):
    return np.array([oracle.ssa_bkl_run(lx, ly, model, rates, init, T, seed, replica=r)[0]
                     for r in range(n)])


@pytest.mark.parametrize("model,rates,lx,ly,T", [
    ("ADSDES", dict(ka=1, kd=1, betaJ=1.0), 3, 3, 0.7),
    ("ISING", dict(ka=1, kd=1, betaJ=0.4), 3, 3, 0.7),
    ("DIFFUSION", dict(ka=0.5, kd=1, betaJ=0.7, nu=2.0), 3, 3, 0.7),
    ("ZGB", dict(yA=0.45, kr=3.0, kd=0.3), 3, 3, 0.8),
    ("ISING1D", dict(ka=1, kd=1, betaJ=1.0, betah=0.5), 8, 1, 0.9),
])
def test_bkl_matches_exponential(model, rates, lx, ly, T):
    base = 3 if model == "ZGB" else 2
    Q = B.generator(lx, ly, model, rates)
    init = (np.zeros(lx * ly, np.uint8) if model == "ZGB"
            else oracle.init_bernoulli(lx, ly, 11, 0.5))
    p0 = B.point_mass(lx, ly, base, init)
    codes = B.codes_of(_bkl_ensemble(lx, ly, model, rates, init, T, 4321, M), base)
    assert chisq_pvalue(codes, B.evolve(p0, Q, T)) > P_OK
    assert chisq_pvalue(codes, B.evolve(p0, Q, 0.8 * T)) < P_OK  # power: a wrong time is rejected


@pytest.mark.parametrize("model,rates", [
    ("ZGB", dict(yA=0.52, kr=10.0, kd=0.1)),
    ("DIFFUSION", dict(ka=1.0, kd=1.0, betaJ=1.0, nu=5.0)),
    ("ISING", dict(ka=1.0, kd=1.0, betaJ=0.4407)),
])
def test_bkl_observables_equal_direct_form(model, rates):
    """Coverage of every state and G(1) after T on 16x16, 300 replicas of
    each form: the means agree within 4 standard errors."""
    lx = ly = 16
    T, n = 1.0, 300
    init = (np.zeros(lx * ly, np.uint8) if model == "ZGB" else oracle.init_bernoulli(lx, ly, 2, 0.5))

    def stats(lat):
        cov, _, pc = oracle.observables(lx, ly, model, lat, 1)
        return np.concatenate([cov, pc])

    a = np.array([stats(l) for l in _bkl_ensemble(lx, ly, model, rates, init, T, 77, n)])
    b = np.array([stats(oracle.ssa_run(lx, ly, model, rates, init, T, 78, replica=r)[0]) for r in range(n)])
    se = np.sqrt(a.var(axis=0, ddof=1) / n + b.var(axis=0, ddof=1) / n) + 1e-12
    z = np.abs(a.mean(axis=0) - b.mean(axis=0)) / se
    assert np.all(z < 4), z

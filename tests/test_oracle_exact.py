"""Pin the oracle's SSA and FS schemes to exact laws on tiny lattices.

Serial SSA vs e^{TQ} (Eq. generator, Eq. semigroup); FS Lie / Strang /
random schedules vs the exact operator products of Eq. lie, Eq. strang and
Eq. SLPCS built from the E/O split of the generator (Eq. opdecomp). The law
of the final state over many independent replicas is tested by chi-square.
Each test also checks that the same samples reject a wrong law (power)."""
import numpy as np
import pytest

import oracle
import oracle.brute as B
from stats_util import chisq_pvalue

M = 20000
P_OK = 1e-3


@pytest.mark.parametrize("model,rates,lx,ly,T", [
    ("ADSDES", dict(ka=1, kd=1, betaJ=1.0), 3, 3, 0.7),
    ("ISING", dict(ka=1, kd=1, betaJ=0.4), 3, 3, 0.7),
    ("DIFFUSION", dict(ka=0.5, kd=1, betaJ=0.7, nu=2.0), 3, 3, 0.7),
    ("ZGB", dict(yA=0.45, kr=3.0, kd=0.3), 3, 3, 0.8),
])
def test_ssa_matches_exponential(model, rates, lx, ly, T):
    base = 3 if model == "ZGB" else 2
    Q = B.generator(lx, ly, model, rates)
    init = (np.zeros(lx * ly, np.uint8) if model == "ZGB"
            else oracle.init_bernoulli(lx, ly, 11, 0.5))
    p0 = B.point_mass(lx, ly, base, init)
    samp = oracle.ssa_ensemble(lx, ly, model, rates, T, 1234, M, init)
    codes = B.codes_of(samp, base)
    assert chisq_pvalue(codes, B.evolve(p0, Q, T)) > P_OK
    # power: a law at a different time is rejected
    assert chisq_pvalue(codes, B.evolve(p0, Q, 0.8 * T)) < P_OK


SCHEMES = {"LIE": B.lie, "STRANG": B.strang, "RANDOM": B.random_sl_mean,
           "RANDOM_ORDER": B.random_order_mean}


@pytest.mark.parametrize("model,rates", [
    ("ADSDES", dict(ka=1, kd=2, betaJ=2.0)),
    ("ISING", dict(ka=1, kd=1, betaJ=0.5)),
    ("ZGB", dict(yA=0.45, kr=3.0, kd=0.3)),
])
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_fs_matches_operator_product_2x4(model, rates, scheme):
    # 2x4 periodic lattice, 1x2 cells: 2 E and 2 O cells
    lx, ly, qx, qy = 2, 4, 1, 2
    base = 3 if model == "ZGB" else 2
    QE = B.generator(lx, ly, model, rates, qx, qy, 0)
    QO = B.generator(lx, ly, model, rates, qx, qy, 1)
    init = (np.zeros(lx * ly, np.uint8) if model == "ZGB"
            else oracle.init_bernoulli(lx, ly, 5, 0.5))
    p0 = B.point_mass(lx, ly, base, init)
    dt, n = 0.5, 2
    samp = oracle.fs_ensemble(lx, ly, qx, qy, model, rates, scheme, dt, dt * n, 77, M, init)
    codes = B.codes_of(samp, base)
    assert chisq_pvalue(codes, SCHEMES[scheme](p0, QE, QO, dt, n)) > P_OK
    if scheme == "LIE":
        # power: the product with the colours swapped is rejected
        assert chisq_pvalue(codes, B.lie(p0, QO, QE, dt, n)) < P_OK
    if scheme == "STRANG":
        # power: a Lie product (half steps not taken) is rejected
        assert chisq_pvalue(codes, B.lie(p0, QE, QO, dt, n)) < P_OK


@pytest.mark.parametrize("scheme", ["LIE", "STRANG"])
def test_fs_matches_operator_product_4x4(scheme):
    # 4x4 periodic, 2x2 cells (the smallest lattice the CUDA library accepts);
    # 65536 states, bins pooled below 5 expected counts
    lx, ly, qx, qy = 4, 4, 2, 2
    rates = dict(ka=1, kd=1, betaJ=0.6)
    QE = B.generator(lx, ly, "ISING", rates, qx, qy, 0)
    QO = B.generator(lx, ly, "ISING", rates, qx, qy, 1)
    init = oracle.init_bernoulli(lx, ly, 9, 0.5)
    p0 = B.point_mass(lx, ly, 2, init)
    dt, n = 0.2, 2
    samp = oracle.fs_ensemble(lx, ly, qx, qy, "ISING", rates, scheme, dt, dt * n, 3, M, init)
    codes = B.codes_of(samp, 2)
    assert chisq_pvalue(codes, SCHEMES[scheme](p0, QE, QO, dt, n)) > P_OK
    wrong = B.lie(p0, QO, QE, dt, n) if scheme == "LIE" else B.lie(p0, QE, QO, dt, n)
    assert chisq_pvalue(codes, wrong) < P_OK


def test_diffusion_frozen_halo_window():
    """One E window of the diffusion model from a fixed snapshot: each E cell's
    write set follows its own CTMC with rates read from the snapshot outside
    the write set (the frozen-halo reading of Step 1 for two-site events)."""
    lx, ly, qx, qy = 8, 4, 2, 2
    rates = dict(ka=0.5, kd=1.0, betaJ=0.8, nu=3.0)
    snap = oracle.init_bernoulli(lx, ly, 21, 0.5)
    h = 0.3
    ncx = lx // qx
    cells = [m for m in range(ncx * (ly // qy)) if ((m % ncx) + (m // ncx)) % 2 == 0][:2]
    outs = np.zeros((M, lx * ly), np.uint8)
    for r in range(M):
        run = oracle.FSRun(lx, ly, qx, qy, "DIFFUSION", rates, snap, replica=r)
        run.window(0, h, seed=31, w=0)
        outs[r] = run.lat
    for m in cells:
        ws, p = B.window_frozen_halo(lx, ly, qx, qy, "DIFFUSION", rates, snap, 0, h, m)
        codes = B.codes_of(outs[:, ws], 2)
        assert chisq_pvalue(codes, p) > P_OK
        # power: the law under the full (unfrozen) dynamics of this cell differs
        ws2, p_long = B.window_frozen_halo(lx, ly, qx, qy, "DIFFUSION", rates, snap, 0,
                                           1.5 * h, m)
        assert chisq_pvalue(codes, p_long) < P_OK

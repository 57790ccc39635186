"""Pin the 1D Ising ring (Section 7, the benchmark with Eq. exactcov1d and
Eq. exactcorr1d): the ring's rates against its Hamiltonian (detailed
balance of the brute-force generator), the transfer-matrix closed forms
against brute-force Gibbs sums, the oracle's windows against the exact
operator products on an 8-site ring, and a long oracle run against the
infinite-ring coverage and correlation."""
import math

import numpy as np
import pytest

import oracle
import oracle.brute as B
from oracle import closed_forms as CF
from stats_util import chisq_pvalue

M = 20000
P_OK = 1e-3


def test_brute_generator_is_gibbs_balanced():
    """pi Q = 0 with pi the Gibbs measure of H = -K sum s s' + h sum s
    (reading of the sign of h in the Arrhenius exponent, as in 2D)."""
    for bK, bh, ka, kd in [(1.3, 0.4, 1.0, 1.0), (-0.7, 1.1, 1.0, 1.0), (2.0, 0.5, 0.6, 1.5)]:
        rates = dict(ka=ka, kd=kd, betaJ=bK, betah=bh)
        Q = B.generator(8, 1, "ISING1D", rates).toarray()
        g = B.gibbs_ising1d(8, bK, bh, ka, kd)
        assert np.abs(g @ Q).max() < 1e-12
        # power: the measure with the field's sign flipped is not stationary
        assert np.abs(B.gibbs_ising1d(8, bK, -bh, ka, kd) @ Q).max() > 1e-3


@pytest.mark.parametrize("bK,bh", [(1.0, 0.5), (2.0, 1.0), (4.0, 1.0), (1.0, 3.0), (-1.0, 0.2)])
def test_transfer_matrix_matches_gibbs_sum(bK, bh):
    L = 8
    g = B.gibbs_ising1d(L, bK, bh)
    S = B.decode(L, 1, 2).astype(np.float64)
    cov, corr = CF.ising1d_ring(L, bK, bh, 3)
    assert cov == pytest.approx(float(g @ S[:, 0]), abs=1e-13)
    for r in range(1, 4):
        assert corr[r - 1] == pytest.approx(float(g @ (S[:, 0] * S[:, r])), abs=1e-13)
    # the infinite-ring forms are the long-ring limits of the same sums
    cov_l, corr_l = CF.ising1d_ring(4096, bK, bh, 3)
    th = CF.ising1d_coverage(bK, bh)
    assert th == pytest.approx(cov_l, abs=1e-12)
    for r in range(1, 4):
        assert CF.ising1d_covariance(bK, bh, r) == pytest.approx(corr_l[r - 1] - th * th,
                                                                 abs=1e-12)


def test_printed_field_sign_reading():
    """Eq. exactcov1d with h' = beta (h - K)/2 as printed gives coverage below
    1/2 at h = 0 with attractive K, where the exact ring sum is above 1/2; the
    reading h' = beta (K - h)/2 is the one that matches."""
    bK = 2.0
    exact = CF.ising1d_ring(64, bK, 0.0)[0]
    assert exact > 0.5
    assert CF.ising1d_coverage(bK, 0.0) == pytest.approx(exact, abs=1e-12)
    hp_printed = 0.5 * (0.0 - bK)
    printed = 0.5 * (1 + math.sinh(hp_printed) / math.sqrt(math.sinh(hp_printed) ** 2
                                                            + math.exp(-bK)))
    assert printed < 0.5


def test_rates_and_total_rate():
    rates = dict(ka=0.8, kd=1.3, betaJ=1.7, betah=0.6)
    r = oracle.rates("ISING1D", **rates)
    assert len(r) == 6
    for n in range(3):
        assert r[n] == 0.8
        assert r[3 + n] == pytest.approx(1.3 * math.exp(-(1.7 * n - 0.6)), rel=1e-15)
    L = 8
    Q = B.generator(L, 1, "ISING1D", rates)
    S = B.decode(L, 1, 2)
    exit_rate = -Q.diagonal()
    for code in range(0, len(S), 3):
        lam, _ = oracle.total_rate(L, 1, "ISING1D", rates, S[code].astype(np.uint8))
        assert lam == pytest.approx(exit_rate[code], rel=1e-12)


def test_ring_cells_partition_sites():
    L, q = 24, 3
    lat = np.zeros(L, np.uint8)
    seen = []
    for m in range(L // q):
        col = m % 2
        o, t, k, _ = oracle.cell_members(L, 1, q, 1, "ISING1D", dict(betaJ=1.0), lat, m, col)
        assert np.all(k == 0)
        seen += o.tolist()
        assert sorted(oracle.cell_writeset(L, 1, q, 1, "ISING1D", m, col).tolist()) == \
            list(range(m * q, (m + 1) * q))
    assert sorted(seen) == list(range(L))


def test_ring_geometry_rules():
    lat = np.zeros(16, np.uint8)
    with pytest.raises(ValueError):  # qy must be 1 on a ring
        oracle.FSRun(8, 2, 2, 2, "ISING1D", dict(betaJ=1.0), np.zeros(16, np.uint8)).run(
            "LIE", 0.1, 0.1, 1)
    with pytest.raises(ValueError):  # L must be a multiple of 2q
        oracle.FSRun(12, 1, 4, 1, "ISING1D", dict(betaJ=1.0), lat[:12]).run("LIE", 0.1, 0.1, 1)


def test_ssa_matches_exponential_ring():
    L, T = 8, 0.7
    rates = dict(ka=1.0, kd=1.0, betaJ=1.2, betah=0.3)
    Q = B.generator(L, 1, "ISING1D", rates)
    init = oracle.init_bernoulli(L, 1, 11, 0.5)
    p0 = B.point_mass(L, 1, 2, init)
    codes = B.codes_of(oracle.ssa_ensemble(L, 1, "ISING1D", rates, T, 99, M, init), 2)
    assert chisq_pvalue(codes, B.evolve(p0, Q, T)) > P_OK
    assert chisq_pvalue(codes, B.evolve(p0, Q, 0.8 * T)) < P_OK


SCHEMES = {"LIE": B.lie, "STRANG": B.strang, "RANDOM": B.random_sl_mean,
           "RANDOM_ORDER": B.random_order_mean}


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_fs_matches_operator_product_ring(scheme):
    # 8-site ring, 2-site cells: 2 E and 2 O cells
    L, q = 8, 2
    rates = dict(ka=1.0, kd=1.0, betaJ=2.0, betah=0.5)
    QE = B.generator(L, 1, "ISING1D", rates, q, 1, 0)
    QO = B.generator(L, 1, "ISING1D", rates, q, 1, 1)
    init = oracle.init_bernoulli(L, 1, 5, 0.5)
    p0 = B.point_mass(L, 1, 2, init)
    dt, n = 0.5, 2
    codes = B.codes_of(oracle.fs_ensemble(L, 1, q, 1, "ISING1D", rates, scheme, dt, dt * n,
                                          31, M, init), 2)
    assert chisq_pvalue(codes, SCHEMES[scheme](p0, QE, QO, dt, n)) > P_OK
    if scheme == "LIE":
        assert chisq_pvalue(codes, B.lie(p0, QO, QE, dt, n)) < P_OK
    if scheme == "STRANG":
        assert chisq_pvalue(codes, B.lie(p0, QE, QO, dt, n)) < P_OK


def test_long_run_matches_infinite_ring():
    """Time-averaged coverage and nearest-neighbour covariance of an oracle
    Lie run on a 2048-site ring at small dt against Eq. exactcov1d and
    Eq. exactcorr1d (with the sign reading above). Batch means give the error."""
    L, q, bK, bh = 2048, 16, 2.0, 1.0
    rates = dict(ka=1.0, kd=1.0, betaJ=bK, betah=bh)
    run = oracle.FSRun(L, 1, q, 1, "ISING1D", rates, oracle.init_bernoulli(L, 1, 3, 0.5))
    run.run("LIE", 0.05, 20.0, 7)
    covs, c1s = [], []
    for _ in range(120):
        run.run("LIE", 0.05, 0.5, 7)
        cov, _, pc = oracle.observables(L, 1, "ISING1D", run.lat, 1)
        covs.append(cov[1])
        c1s.append(pc[0] - cov[1] ** 2)
    covs, c1s = np.array(covs), np.array(c1s)
    bm = covs.reshape(12, 10).mean(axis=1)
    se = bm.std(ddof=1) / math.sqrt(len(bm))
    want = CF.ising1d_coverage(bK, bh)
    assert abs(covs.mean() - want) < max(5 * se, 3e-3), (covs.mean(), want, se)
    bm1 = c1s.reshape(12, 10).mean(axis=1)
    se1 = bm1.std(ddof=1) / math.sqrt(len(bm1))
    want1 = CF.ising1d_covariance(bK, bh, 1)
    assert abs(c1s.mean() - want1) < max(5 * se1, 3e-3), (c1s.mean(), want1, se1)
    # power: the printed sign of the field would put the coverage elsewhere
    assert abs(covs.mean() - (1 - want)) > 0.1

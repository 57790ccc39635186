"""The 1D Ising ring on the GPU (Section 7, Eq. exactcov1d, Eq. exactcorr1d):
bit-identical windows against the oracle for ring cells of 1..1024 sites
(ragged cells included), both engines and bit-packed storage; then the
paper's benchmark -- rings of N = 2^15 sites at dt = 1.0, a batch of
(beta, h) points -- against the transfer-matrix coverage and two-point
correlation."""
import math

import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from gpu_util import gpu_ctx, match_oracle
from oracle import closed_forms as CF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _rates(beta, h, K=1.0):
    return dict(ka=1.0, kd=1.0, betaJ=beta * K, betah=beta * h)


# (L, q): tiny, ragged (q not a power of two), one-lane and 32-lane cells
RINGS = [(8, 2), (96, 6), (192, 3), (2048, 32), (6000, 1000), (4096, 1024), (4096, 512)]


def _bit_exact(L, q, rates, scheme, dt, T, seed, engine="PLAIN", bitpacked=False):
    init = oracle.init_bernoulli(L, 1, seed, 0.5)
    orc = oracle.FSRun(L, 1, q, 1, "ISING1D", rates, init).run(scheme, dt, T, seed)
    c = F.Context(L, 1, "ISING1D", rates, (q, 1), bitpacked=bitpacked)
    with c:
        c.set_engine(engine)
        c.set_state(init)
        c.run(scheme, dt, T, seed)
        g, st, wl = c.get_state(), c.stats(), c.workload()
    match_oracle((g, st["events"], wl), orc,
                 lambda: gpu_ctx(L, 1, (q, 1), "ISING1D", rates, init, engine=engine, packed=bitpacked),
                 lambda: oracle.FSRun(L, 1, q, 1, "ISING1D", rates, init), scheme, dt, T, seed,
                 what=f"ring {L} q={q} {scheme} {engine}")
    assert st["events"] > 0


@pytest.mark.parametrize("L,q", RINGS)
@pytest.mark.parametrize("scheme", ["LIE", "STRANG", "RANDOM", "RANDOM_ORDER"])
def test_ring_bit_exact(L, q, scheme):
    _bit_exact(L, q, _rates(2.0, 0.5), scheme, 0.25, 2.0, 0x1D + L + q)


@pytest.mark.parametrize("L,q", [(2048, 32), (4096, 1024), (6000, 1000)])
@pytest.mark.parametrize("scheme", ["LIE", "RANDOM"])
def test_ring_persistent_bit_exact(L, q, scheme):
    _bit_exact(L, q, _rates(1.0, 1.5), scheme, 0.5, 3.0, 0xABC + q, engine="PERSISTENT")


@pytest.mark.parametrize("L,q,engine", [(2048, 32, "PLAIN"), (2048, 16, "PERSISTENT"),
                                        (4096, 1024, "PLAIN"), (4096, 1024, "PERSISTENT"),
                                        (1536, 96, "PLAIN")])
def test_ring_bitpacked_bit_exact(L, q, engine):
    _bit_exact(L, q, _rates(4.0, 1.0), "STRANG", 0.5, 3.0, 0x51 + q, engine=engine,
               bitpacked=True)


def test_ring_full_size_bit_exact():
    """The benchmark ring itself (N = 2^15, dt = 1.0, Lie) for 8 steps, at
    the cell length the autotuner picks, against the oracle."""
    L = 1 << 15
    rates = _rates(2.0, 0.5)
    init = oracle.init_bernoulli(L, 1, 3, 0.5)
    with F.Context(L, 1, "ISING1D", rates, None) as c:
        qx = c.info()["qx"]
        c.set_engine("PERSISTENT")
        c.set_state(init)
        c.run("LIE", 1.0, 8.0, 99)
        got = (c.get_state(), c.stats()["events"], c.workload())
    orc = oracle.FSRun(L, 1, qx, 1, "ISING1D", rates, init).run("LIE", 1.0, 8.0, 99)
    match_oracle(got, orc, lambda: gpu_ctx(L, 1, (qx, 1), "ISING1D", rates, init, engine="PERSISTENT"),
                 lambda: oracle.FSRun(L, 1, qx, 1, "ISING1D", rates, init), "LIE", 1.0, 8.0, 99,
                 what="2^15 ring")


def test_ring_observables_bit_exact():
    L = 4096
    lat = oracle.init_bernoulli(L, 1, 8, 0.4)
    with F.Context(L, 1, "ISING1D", _rates(1.0, 0.0), (32, 1)) as c:
        c.set_state(lat)
        for rmax in (0, 1, 40):
            cov, en, pc = c.observables(0, rmax)
            ocov, oen, opc = oracle.observables(L, 1, "ISING1D", lat, rmax)
            assert np.array_equal(cov, ocov) and en == oen and np.array_equal(pc, opc)
            assert not pc[rmax:].any()  # a ring has no vertical pairs


BETAS = (1.0, 2.0, 4.0)
HS = (0.0, 0.5, 1.0, 1.5, 2.0)


def test_phase_diagram_and_correlation_n2_15():
    """Figs. phase1D and spcorr1D: mean coverage over a batch of rings of
    N = 2^15 sites at dt = 1.0 (Lie, K = 1) for beta in {1, 2, 4} and
    h in [0, 2], against Eq. exactcov1d; the two-point correlation at
    h = 1 against Eq. exactcorr1d. Time averages after a burn-in; batch
    means give the standard error, and the allowance 0.005 covers the
    splitting bias at dt = 1.0."""
    L, rmax = 1 << 15, 8
    pts = [(b, h) for b in BETAS for h in HS]
    batch = [dict(lx=L, ly=1, rates=_rates(b, h)) for b, h in pts]
    cov = [[] for _ in pts]
    corr = [[] for _ in pts]
    with F.Context(model="ISING1D", q=None, batch=batch) as c:
        c.set_engine("PERSISTENT")
        c.init_random(2024, 0.5)
        c.run("LIE", 1.0, 50.0, 7)
        for _ in range(200):
            c.run("LIE", 1.0, 1.0, 7)
            for i in range(len(pts)):
                cv, _, pc = c.observables(i, rmax)
                cov[i].append(cv[1])
                corr[i].append(pc[:rmax])
    for i, (b, h) in enumerate(pts):
        x = np.array(cov[i])
        bm = x.reshape(20, 10).mean(axis=1)
        se = bm.std(ddof=1) / math.sqrt(len(bm))
        want = CF.ising1d_coverage(b, b * h)
        assert abs(x.mean() - want) < 5 * se + 0.005, (b, h, x.mean(), want, se)
        if abs(want - 0.5) > 0.05:
            # the printed sign of the field would give 1 - want
            assert abs(x.mean() - (1.0 - want)) > 0.05
        if h == 1.0:
            g = np.array(corr[i])                     # (samples, rmax)
            gm = g.reshape(20, 10, rmax).mean(axis=1)  # batch means
            seg = gm.std(axis=0, ddof=1) / math.sqrt(20)
            th = CF.ising1d_coverage(b, b * h)
            for r in range(1, rmax + 1):
                want_g = CF.ising1d_covariance(b, b * h, r) + th * th
                assert abs(g[:, r - 1].mean() - want_g) < 5 * seg[r - 1] + 0.01, (b, r)


def _coverage_paths(dt, M, T, start, seed):
    """Coverage of M independent rings of 2^15 sites (beta = 4, h = 1, K = 1)
    sampled once per time unit for T units."""
    L = 1 << 15
    batch = [dict(lx=L, ly=1, rates=_rates(4.0, 1.0)) for _ in range(M)]
    S = np.zeros((T + 1, M))
    with F.Context(model="ISING1D", q=(1024, 1), batch=batch) as c:
        c.set_engine("PERSISTENT")
        c.set_clock("FP32")
        c.init_random(seed, start)
        S[0] = [c.observables(r, 0)[0][1] for r in range(M)]
        for k in range(1, T + 1):
            c.run("LIE", dt, 1.0, seed)
            S[k] = [c.observables(r, 0)[0][1] for r in range(M)]
    return S


def _autocorr(S, burn, lags):
    X = S[burn:] - S[burn:].mean(axis=0)
    v = (X * X).mean()
    return np.array([(X[:len(X) - k] * X[k:]).mean() / v for k in lags])


def test_coverage_process_converges_in_dt():
    """Fig. samples1D: the total-coverage process of 256 realisations at
    beta = 4, h = 1 on N = 2^15 (binary32 clock). Its mean and spread along
    the relaxation from the empty lattice, and its autocorrelation in
    equilibrium, at dt = 1.0 and 0.1 against dt = 0.01 (the serial-SSA
    limit of the splitting). Means by z-score; the autocorrelation within
    0.05."""
    M, T = 256, 40
    ref = _coverage_paths(0.01, M, T, 0.0, 31)
    for dt in (1.0, 0.1):
        S = _coverage_paths(dt, M, T, 0.0, 32 if dt == 1.0 else 33)
        se = np.sqrt(S[1:].var(axis=1, ddof=1) / M + ref[1:].var(axis=1, ddof=1) / M)
        z = (S[1:].mean(axis=1) - ref[1:].mean(axis=1)) / se
        assert np.abs(z).max() < 4.5, (dt, z)
        # spread across realisations within 25% of the reference
        ratio = S[5:].std(axis=1) / ref[5:].std(axis=1)
        assert np.all(np.abs(ratio - 1) < 0.25), (dt, ratio)
    lags = [0, 1, 2, 5, 10, 20]
    acs = {}
    for dt, seed in ((0.01, 41), (0.1, 42), (1.0, 43)):
        acs[dt] = _autocorr(_coverage_paths(dt, M, 300, 0.5, seed), 100, lags)
    assert acs[0.01][1] > 0.3  # the process is visibly correlated over one time unit
    for dt in (0.1, 1.0):
        assert np.abs(acs[dt] - acs[0.01]).max() < 0.05, (dt, acs[dt], acs[0.01])

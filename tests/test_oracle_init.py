"""Pins of the oracle's initial states against the laws that define them
(not against the oracle itself): the Bernoulli(p) random start of the
benchmarks (Section 7's random initial configurations) and the seeded
Gaussian-bump pre-coverage of the catalysis workload (reading 13: species A
with probability amp * g(dx) * g(dy), g(d) = exp(-d^2 / 2 s^2), periodic
distance to a centre drawn from the counter-based generator)."""
import numpy as np
import pytest
from scipy import stats

import oracle


@pytest.mark.parametrize("p", [0.0, 1.0, 0.1, 0.37, 0.5, 0.9])
def test_bernoulli_coverage_matches_p(p):
    """Coverage of 2^20 sites against p by a z-test (5 standard errors);
    p = 0 and p = 1 give the empty and the full lattice exactly."""
    lx = ly = 1024
    lat = oracle.init_bernoulli(lx, ly, 0xB0 + int(100 * p), p)
    assert set(np.unique(lat)) <= {0, 1}
    if p in (0.0, 1.0):
        assert np.all(lat == int(p))
        return
    n = lat.size
    z = (lat.mean() - p) / np.sqrt(p * (1 - p) / n)
    assert abs(z) < 5, z


def test_bernoulli_threshold_resolution():
    """Coverage follows p on a fine grid of p (a threshold off by a factor
    of two, or taken on another output word with a bias, fails here)."""
    lx, ly = 512, 512
    for p in (0.01, 0.2, 0.49, 0.51, 0.75, 0.99):
        lat = oracle.init_bernoulli(lx, ly, 7, p)
        z = (lat.mean() - p) / np.sqrt(p * (1 - p) / lat.size)
        assert abs(z) < 5, (p, z)


def test_bernoulli_sites_are_independent():
    """Nearest-neighbour pairs are occupied with probability p^2, and the
    lattices of two replicas (or two seeds) are independent of each other."""
    lx = ly = 1024
    p = 0.37
    a = oracle.init_bernoulli(lx, ly, 11, p).reshape(ly, lx).astype(np.float64)
    b = oracle.init_bernoulli(lx, ly, 11, p, replica=1).reshape(ly, lx).astype(np.float64)
    c = oracle.init_bernoulli(lx, ly, 12, p).reshape(ly, lx).astype(np.float64)
    n = a.size
    se = np.sqrt(p * p * (1 - p * p) / n)
    for pair in (a * np.roll(a, 1, 1), a * np.roll(a, 1, 0), a * b, a * c):
        assert abs(pair.mean() - p * p) < 5 * se
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def _bump_law(lx, ly, x0, y0, amp, width):
    """amp * g(dx) * g(dy) on the periodic lattice, written out in numpy."""
    dx = np.abs(np.arange(lx) - x0)
    dx = np.minimum(dx, lx - dx)
    dy = np.abs(np.arange(ly) - y0)
    dy = np.minimum(dy, ly - dy)
    gx = np.exp(-dx.astype(np.float64) ** 2 / (2 * width ** 2))
    gy = np.exp(-dy.astype(np.float64) ** 2 / (2 * width ** 2))
    return amp * gy[:, None] * gx[None, :]


def _centre(lx, ly, seed, rep=0):
    """The bump's centre: words 0 and 1 of the generator at counter
    (0, 2^32 - 1, 0, replica | 3 << 24) under the seed, modulo the sides."""
    o = oracle.philox([0, 0xFFFFFFFF, 0, rep | (3 << 24)], [seed & 0xFFFFFFFF, seed >> 32])
    return int(o[0]) % lx, int(o[1]) % ly


def _chi2_rows_cols(lat, p):
    """Chi-square of the per-row and per-column occupancy against the law p
    (independent sites: variance sum p(1-p)); rows/columns with expected
    count below 5 are pooled out. Returns the two survival probabilities."""
    out = []
    for axis in (1, 0):
        obs = lat.sum(axis=axis)
        exp = p.sum(axis=axis)
        var = (p * (1 - p)).sum(axis=axis)
        keep = exp > 5
        chi = float((((obs - exp) ** 2)[keep] / var[keep]).sum())
        out.append(stats.chi2.sf(chi, int(keep.sum())))
    return out


@pytest.mark.parametrize("lx,ly,amp,width,species,rep", [
    (1024, 768, 0.9, 1024 / 8, 1, 0),
    (512, 512, 0.6, 40.0, 2, 3),
    (2048, 256, 0.9, 2048 / 8, 1, 1),
])
def test_bump_follows_the_gaussian_law(lx, ly, amp, width, species, rep):
    seed = 0x5EED0004
    lat = oracle.init_bump(lx, ly, seed, amp, width, species, replica=rep)
    assert set(np.unique(lat)) <= {0, species}
    occ = (lat.reshape(ly, lx) == species).astype(np.float64)
    x0, y0 = _centre(lx, ly, seed, rep)
    p = _bump_law(lx, ly, x0, y0, amp, width)
    p_rows, p_cols = _chi2_rows_cols(occ, p)
    assert p_rows > 1e-4 and p_cols > 1e-4, (p_rows, p_cols)
    # total occupancy against its expectation
    z = (occ.sum() - p.sum()) / np.sqrt((p * (1 - p)).sum())
    assert abs(z) < 5, z
    # the centre read back from the data: circular mean of the occupied
    # sites' coordinates, within two sites of the drawn centre
    ys, xs = np.nonzero(occ)
    for coords, L, c in ((xs, lx, x0), (ys, ly, y0)):
        ang = 2 * np.pi * coords / L
        est = (np.arctan2(np.sin(ang).mean(), np.cos(ang).mean()) * L / (2 * np.pi)) % L
        d = abs(est - c)
        assert min(d, L - d) < 2.0, (est, c)


def test_bump_statistic_rejects_a_wrong_law():
    """Power of the statistic above: the same lattice against a law with
    the width 10% off, the amplitude 5% off or the centre moved by 8 sites
    is rejected."""
    lx, ly, amp, width = 1024, 768, 0.9, 128.0
    seed = 0x5EED0004
    occ = (oracle.init_bump(lx, ly, seed, amp, width, 1).reshape(ly, lx) == 1).astype(np.float64)
    x0, y0 = _centre(lx, ly, seed)
    for law in (_bump_law(lx, ly, x0, y0, amp, width * 1.1),
                _bump_law(lx, ly, x0, y0, amp * 0.95, width),
                _bump_law(lx, ly, (x0 + 8) % lx, y0, amp, width)):
        assert min(_chi2_rows_cols(occ, law)) < 1e-6

"""Pin the oracle's integer observables to a numpy recount."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("lx,ly,nstates", [(8, 8, 2), (16, 12, 3), (4, 4, 2)])
def test_observables_recount(lx, ly, nstates):
    rng = np.random.default_rng(lx * ly)
    lat = rng.integers(0, nstates, size=(ly, lx)).astype(np.uint8)
    rmax = 3
    counts, pairs, gx, gy = oracle.observables_int(lx, ly, lat, rmax)
    one = (lat == 1).astype(np.int64)
    assert counts[:nstates].tolist() == np.bincount(lat.ravel(), minlength=3)[:nstates].tolist()
    assert pairs == int((one * np.roll(one, -1, 1)).sum() + (one * np.roll(one, -1, 0)).sum())
    for r in range(1, rmax + 1):
        assert gx[r - 1] == int((one * np.roll(one, -r, 1)).sum())
        assert gy[r - 1] == int((one * np.roll(one, -r, 0)).sum())


def test_ising_energy_all_up_and_checkerboard():
    lx = ly = 8
    cov, e, _ = oracle.observables(lx, ly, "ISING", np.ones(lx * ly, np.uint8), 1)
    assert cov[1] == 1.0 and e == -2.0  # every bond aligned: -2 per site
    x, y = np.meshgrid(np.arange(lx), np.arange(ly))
    cov, e, _ = oracle.observables(lx, ly, "ISING", ((x + y) % 2).astype(np.uint8), 1)
    assert e == 2.0

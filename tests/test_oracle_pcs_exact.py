"""Processor communication schedules compared on exact laws (Section 4.1):
the bias of the mean coverage against the exact e^{TL}, computed from the
exact operator products on a 4x4 lattice (65,536 states) from the uniform
initial law, for 1x1 and 2x2 cells. What the paper states, and these pin
independently of any sampling:
- the Lie schedule's error lives on cell boundaries and shrinks as the cells
  grow (Eq. liebound): fewer boundary bonds, smaller bias;
- the random sub-lattice schedule's error does not depend on the cell size
  to leading order (Eq. randomtimestep) and is first order in dt;
- at equal tolerance Lie admits a window several times larger (Eq.
  pcscompare): its bias at dt = 1 is far below the random schedule's at
  dt = 1/4.
The same exact values are the yardstick of the GPU check in
tests/test_gpu_pcs_exact.py."""
import numpy as np
import pytest

import oracle.brute as B

L, T = 4, 2.0
RATES = dict(ka=1.0, kd=1.0, betaJ=2.0)


def exact_biases():
    """{(q, scheme, dt): mean coverage under the schedule's law minus under
    e^{TL}}, plus the exact mean itself under key 'exact'."""
    S = B.decode(L, L, 2)
    f = (S == 1).mean(axis=1)
    p0 = np.full(1 << (L * L), 1.0 / (1 << (L * L)))
    exact = B.evolve(p0, B.generator(L, L, "ADSDES", RATES), T) @ f
    out = {"exact": exact}
    for q in (1, 2):
        QE = B.generator(L, L, "ADSDES", RATES, q, q, 0)
        QO = B.generator(L, L, "ADSDES", RATES, q, q, 1)
        out[q, "LIE", 1.0] = B.lie(p0, QE, QO, 1.0, 2) @ f - exact
        for dt in (0.25, 0.125):
            out[q, "RANDOM", dt] = B.random_sl_mean(p0, QE, QO, dt, int(round(T / dt))) @ f - exact
    return out


@pytest.fixture(scope="module")
def biases():
    return exact_biases()


def test_lie_bias_shrinks_with_the_cell(biases):
    b1, b2 = biases[1, "LIE", 1.0], biases[2, "LIE", 1.0]
    assert abs(b1) > 1e-3
    assert abs(b2) < 0.5 * abs(b1), (b1, b2)


def test_random_bias_is_order_one_in_the_cell_and_first_order_in_dt(biases):
    r1, r2 = biases[1, "RANDOM", 0.25], biases[2, "RANDOM", 0.25]
    assert abs(r1 - r2) < 0.25 * abs(r1), (r1, r2)
    for q in (1, 2):
        ratio = biases[q, "RANDOM", 0.125] / biases[q, "RANDOM", 0.25]
        assert 0.4 < ratio < 0.6, (q, ratio)


def test_lie_admits_a_larger_window(biases):
    for q in (1, 2):
        assert abs(biases[q, "RANDOM", 0.25]) > 2 * abs(biases[q, "LIE", 1.0])
    assert abs(biases[2, "RANDOM", 0.25]) > 5 * abs(biases[2, "LIE", 1.0])

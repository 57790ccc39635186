"""Pin the oracle's nested (two-level) fractional-step scheme, Section 5
(Eq. sublatt2, Eq. opdecomp2), to what the mathematics fixes:

- the two-level split is a partition of the generator: the four parts
  (super colour, sub colour) sum to L, and each super colour's two parts
  sum to that colour's part of the one-level split (Eq. opdecomp);
- the law of the oracle's final states (chi-square over replicas) equals
  the exact nested operator product on a 4x4 lattice (2x2 super-cells of
  1x1 sub-cells), and rejects both the one-level product (inner splitting
  not taken) and the product with the sub-cell colours swapped;
- as the number of inner steps grows the nested product tends to the
  one-level product over the super-cells (Trotter): error O(1/n_in) for an
  inner Lie splitting, O(1/n_in^2) for an inner Strang splitting;
- with no interaction (betaJ = 0) every part commutes, so every site
  follows its two-state chain exactly: the J = 0 closed form holds on a
  large lattice whatever the schedules.
"""
import numpy as np
import pytest

import oracle
import oracle.brute as B
from oracle import closed_forms as CF
from stats_util import chisq_pvalue

M = 100000
P_OK = 1e-3
RATES = dict(ka=1, kd=1, betaJ=0.3)


@pytest.fixture(scope="module")
def parts():
    Qs = [[B.generator_nested(4, 4, 2, 2, 1, 1, "ISING", RATES, C, c) for c in (0, 1)]
          for C in (0, 1)]
    QE = B.generator(4, 4, "ISING", RATES, 2, 2, 0)
    QO = B.generator(4, 4, "ISING", RATES, 2, 2, 1)
    return Qs, QE, QO


def test_two_level_split_is_a_partition(parts):
    Qs, QE, QO = parts
    Q = B.generator(4, 4, "ISING", RATES)
    assert abs(Qs[0][0] + Qs[0][1] + Qs[1][0] + Qs[1][1] - Q).max() < 1e-12
    assert abs(Qs[0][0] + Qs[0][1] - QE).max() < 1e-12
    assert abs(Qs[1][0] + Qs[1][1] - QO).max() < 1e-12


@pytest.mark.parametrize("scheme,inner,n_in", [("LIE", "LIE", 1), ("LIE", "STRANG", 1),
                                               ("STRANG", "LIE", 2), ("STRANG", "STRANG", 1)])
def test_nested_matches_exact_product(parts, scheme, inner, n_in):
    Qs, QE, QO = parts
    init = oracle.init_bernoulli(4, 4, 9, 0.5)
    p0 = B.point_mass(4, 4, 2, init)
    dt, n = 1.0, 1
    samp = oracle.fs2_ensemble(4, 4, (2, 2), (1, 1), "ISING", RATES, scheme, dt, dt * n, 0x2E5, M,
                               init, inner, n_in)
    codes = B.codes_of(samp, 2)
    assert chisq_pvalue(codes, B.nested_product(p0, Qs, scheme, dt, n, inner, n_in)) > P_OK
    # power: the one-level product over the super-cells, and the nested
    # product with the sub-cell colours swapped, are rejected
    flat = B.lie(p0, QE, QO, dt, n) if scheme == "LIE" else B.strang(p0, QE, QO, dt, n)
    assert chisq_pvalue(codes, flat) < P_OK
    swapped = B.nested_product(p0, [q[::-1] for q in Qs], scheme, dt, n, inner, n_in)
    assert chisq_pvalue(codes, swapped) < P_OK


@pytest.mark.parametrize("inner,order", [("LIE", 1), ("STRANG", 2)])
def test_inner_splitting_tends_to_one_level(parts, inner, order):
    """One outer E window: n_in inner steps against e^{h L^E}."""
    Qs, QE, QO = parts
    p0 = B.point_mass(4, 4, 2, oracle.init_bernoulli(4, 4, 9, 0.5))
    h = 0.5
    exact = B.evolve(p0, QE, h)
    tv = [0.5 * abs(B.nested_window(p0, Qs[0], h, inner, k) - exact).sum() for k in (4, 8)]
    assert abs(np.log2(tv[0] / tv[1]) - order) < 0.3, tv


@pytest.mark.parametrize("scheme,inner,n_in", [("LIE", "STRANG", 3), ("STRANG", "LIE", 2)])
def test_nested_noninteracting_closed_form(scheme, inner, n_in):
    lx = ly = 256
    ka, kd, T = 2.0, 1.0, 1.0
    init = oracle.init_bernoulli(lx, ly, 4, 0.5)
    th0 = init.mean()
    run = oracle.FS2Run(lx, ly, (32, 32), (8, 8), "ADSDES", dict(ka=ka, kd=kd, betaJ=0.0), init)
    run.run(scheme, 0.2, T, 11, inner, n_in)
    got = run.lat.mean()
    want = CF.coverage_noninteracting(T, th0, ka, kd)
    assert abs(got - want) < 4 * np.sqrt(want * (1 - want) / (lx * ly))
    ninner = (2 if inner == "LIE" else 3) * n_in
    nouter = (2 if scheme == "LIE" else 3) * 5
    assert run.windows == nouter * ninner


def test_nested_rejects_bad_geometry():
    init = np.zeros(64 * 64, np.uint8)
    for Q, q, model in (((16, 16), (16, 16), "ISING"),    # one sub-cell per super-cell side
                        ((24, 16), (8, 8), "ISING"),      # odd number of sub-cells across
                        ((16, 16), (8, 8), "ZGB")):       # two-site model
        with pytest.raises(ValueError):
            oracle.FS2Run(64, 64, Q, q, model, RATES, init).run("LIE", 0.1, 0.1, 1)

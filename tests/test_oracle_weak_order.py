"""Pin the exact operator products to the paper's error orders: Lie and the
random sub-lattice schedule are first order in dt (Eq. error and the random
PCS local error of Section 4.1), Strang and the random-order schedule second
order (Eq. error2). Deterministic: exact laws on a 2x4 lattice with 1x2
cells, observable = coverage, T = 1."""
import numpy as np
import pytest

import oracle
import oracle.brute as B

LX, LY, QX, QY = 2, 4, 1, 2
FNS = {"LIE": (B.lie, 1), "STRANG": (B.strang, 2), "RANDOM": (B.random_sl_mean, 1),
       "RANDOM_ORDER": (B.random_order_mean, 2)}


@pytest.mark.parametrize("model,rates", [("ADSDES", dict(ka=1.0, kd=2.0, betaJ=1.0)),
                                         ("ZGB", dict(yA=0.45, kr=3.0, kd=0.3))])
@pytest.mark.parametrize("name", list(FNS))
def test_weak_order(model, rates, name):
    base = 3 if model == "ZGB" else 2
    Q = B.generator(LX, LY, model, rates)
    QE = B.generator(LX, LY, model, rates, QX, QY, 0)
    QO = B.generator(LX, LY, model, rates, QX, QY, 1)
    S = B.decode(LX, LY, base)
    init = (np.zeros(LX * LY, np.uint8) if model == "ZGB"
            else oracle.init_bernoulli(LX, LY, 5, 0.5))
    p0 = B.point_mass(LX, LY, base, init)
    f = (S == 1).mean(axis=1)
    T = 1.0
    exact = B.evolve(p0, Q, T) @ f
    fn, order = FNS[name]
    dts = [0.05, 0.025, 0.0125]
    errs = [abs(fn(p0, QE, QO, dt, int(round(T / dt))) @ f - exact) for dt in dts]
    slope = np.log(errs[-1] / errs[-2]) / np.log(dts[-1] / dts[-2])
    assert abs(slope - order) < 0.15, (errs, slope)

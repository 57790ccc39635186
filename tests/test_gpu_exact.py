"""The CUDA path against exact laws, independently of the oracle.

A batch of 20,000 replicas of a 4x4 periodic Ising lattice (2x2 cells) starts
from independent Bernoulli(1/2) sites (the uniform law on 65,536 states); the
law of the final state over the replicas is compared by chi-square with the
exact operator products of Eq. lie, Eq. strang and Eq. SLPCS built from the
E/O split of the generator (oracle/brute.py, written from the paper's rate
formulas). Both window clocks; the colour-swapped product must be rejected.
Plus Onsager's magnetisation (Eq. exactcov2d) at the 1024^2 benchmark size.
"""
import numpy as np
import pytest

import oracle.brute as B
import paper_1105_4673_gb300 as F
from oracle import closed_forms as CF
from stats_util import chisq_pvalue

pytestmark = pytest.mark.gpu

M = 20000
RATES = dict(ka=1.0, kd=1.0, betaJ=0.6)


@pytest.fixture(scope="module")
def gens():
    from paper_1105_4673_gb300 import build
    build.build()
    QE = B.generator(4, 4, "ISING", RATES, 2, 2, 0)
    QO = B.generator(4, 4, "ISING", RATES, 2, 2, 1)
    p0 = np.full(1 << 16, 1.0 / (1 << 16))
    return QE, QO, p0


def _final_states(scheme, dt, T, clock, engine, seed):
    reps = [dict(lx=4, ly=4, rates=RATES)] * M
    with F.Context(model="ISING", q=(2, 2), batch=reps) as b:
        b.set_clock(clock)
        b.set_engine(engine)
        b.init_random(seed, 0.5)
        b.run(scheme, dt, T, seed)
        assert b.stats()["check_failures"] == 0
        return np.stack([b.get_state(r) for r in range(M)])


FNS = {"LIE": B.lie, "STRANG": B.strang, "RANDOM": B.random_sl_mean,
       "RANDOM_ORDER": B.random_order_mean}


CASES = [(s, c, "PERSISTENT") for s in FNS for c in ("FP64", "FP32")] + [("LIE", "FP64", "PLAIN")]


@pytest.mark.parametrize("scheme,clock,engine", CASES)
def test_gpu_law_matches_exact_product(gens, scheme, clock, engine):
    QE, QO, p0 = gens
    dt, n = 0.2, 2
    states = _final_states(scheme, dt, dt * n, clock, engine, 1234 + len(scheme))
    codes = B.codes_of(states, 2)
    assert chisq_pvalue(codes, FNS[scheme](p0, QE, QO, dt, n)) > 1e-3
    if scheme == "LIE":
        assert chisq_pvalue(codes, B.lie(p0, QO, QE, dt, n)) < 1e-3


def test_onsager_magnetisation_at_benchmark_size():
    """Eq. exactcov2d: below T_c the time-averaged |m| of the 1024^2 lattice
    (16x16 cells, Lie dt = 0.25, binary32 clock, from all spins up) matches
    Onsager's (1 - sinh(2 betaJ)^-4)^(1/8) at betaJ = 0.6."""
    L = 1024
    with F.Context(L, L, "ISING", RATES, (16, 16)) as c:
        c.set_clock("FP32")
        c.set_engine("PERSISTENT")
        c.set_state(np.ones(L * L, np.uint8))
        c.run("LIE", 0.25, 20.0, 5)
        ms = []
        for _ in range(40):
            c.run("LIE", 0.25, 1.0, 5)
            cov = c.observables(0, 0)[0]
            ms.append(abs(2.0 * cov[1] - 1.0))
    assert abs(np.mean(ms) - CF.onsager_magnetisation(0.6)) < 0.005, np.mean(ms)

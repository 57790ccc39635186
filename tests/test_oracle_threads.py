"""The oracle's all-core form (cells of a window spread over threads) is the
same computation as the single-thread run: same-colour cells read only the
window-start snapshot outside their write sets and write disjoint sets
(Eq. exact), so lattices, event counts and workloads are identical."""
import numpy as np
import pytest

import oracle
from workloads import random_lattice

CASES = [
    ("ISING", dict(ka=1.0, kd=1.0, betaJ=0.4407), 128, 64, (16, 16), "LIE", 0.5, 2.0),
    ("ADSDES", dict(ka=1.0, kd=1.0, betaJ=1.0), 64, 64, (8, 8), "RANDOM", 0.1, 1.0),
    ("DIFFUSION", dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0), 64, 64, (8, 8), "RANDOM_ORDER", 0.05, 0.5),
    ("ZGB", dict(yA=0.52, kr=100.0, kd=0.01), 96, 64, (16, 16), "STRANG", 0.02, 0.2),
]


@pytest.mark.parametrize("model,rates,lx,ly,q,scheme,dt,T", CASES)
@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_threads_equal_single_thread(model, rates, lx, ly, q, scheme, dt, T, nthreads):
    init = (random_lattice(lx, ly, 3, 5, p=[0.6, 0.2, 0.2]) if model == "ZGB"
            else oracle.init_bernoulli(lx, ly, 5, 0.4))
    a = oracle.FSRun(lx, ly, *q, model, rates, init).run(scheme, dt, T, 17)
    b = oracle.FSRun(lx, ly, *q, model, rates, init)
    b.run_threads(scheme, dt, T / 2, 17, nthreads)
    b.run_threads(scheme, dt, T / 2, 17, nthreads)  # resumes at the window index
    assert np.array_equal(a.lat, b.lat)
    assert a.events == b.events and a.windows == b.windows and a.events > 0
    assert np.array_equal(a.workload, b.workload)

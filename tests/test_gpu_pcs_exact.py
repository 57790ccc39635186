"""The GPU's schedule biases at matching (cell size, dt) against the exact
values of tests/test_oracle_pcs_exact.py: 2^18 replicas of the 4x4
adsorption/desorption lattice (betaJ = 2) from independent Bernoulli(1/2)
sites (the uniform initial law), advanced to T = 2 in one persistent
binary64 launch; the replica mean of the coverage must equal the exact law's
mean under the schedule (Lie, dt = 1; random sub-lattice, dt = 1/4) within 4
standard errors, for 1x1 and 2x2 cells -- and, where the exact bias exceeds
6 standard errors, differ from the mean under e^{TL} itself."""
import numpy as np
import pytest

import paper_1105_4673_gb300 as F
from test_oracle_pcs_exact import L, RATES, T, exact_biases

pytestmark = pytest.mark.gpu

M, BATCHES = 1 << 16, 4  # 2^18 replicas in batches of the library's largest replica count


@pytest.fixture(scope="module")
def exact():
    from paper_1105_4673_gb300 import build
    build.build()
    return exact_biases()


@pytest.mark.parametrize("q,scheme,dt", [(1, "LIE", 1.0), (2, "LIE", 1.0), (1, "RANDOM", 0.25),
                                         (2, "RANDOM", 0.25)])
def test_gpu_bias_matches_exact(exact, q, scheme, dt):
    reps = [dict(lx=L, ly=L, rates=RATES)] * M
    cov = []
    for k in range(BATCHES):
        with F.Context(model="ADSDES", q=(q, q), batch=reps) as b:
            b.set_engine("PERSISTENT")
            b.init_random(0xB1A5 + 101 * k + q + len(scheme), 0.5)
            b.run(scheme, dt, T, 0xB1A5 + 7 * q + 1000 * k)
            assert b.stats()["check_failures"] == 0
            cov += [b.observables(r, 0)[0][1] for r in range(M)]
    cov = np.array(cov)
    mean, se = cov.mean(), cov.std(ddof=1) / np.sqrt(len(cov))
    want = exact["exact"] + exact[q, scheme, dt]
    assert abs(mean - want) < 4 * se, (mean, want, se)
    if abs(exact[q, scheme, dt]) > 6 * se:
        assert abs(mean - exact["exact"]) > 3 * se

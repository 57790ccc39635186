"""Bit-packed lattices (1 bit per site in device memory) give exactly the
results of the byte-per-site layout: bit-identical to the oracle with the
binary64 clock, bitwise equal to the unpacked form with the binary32 clock,
for cells narrower than a word (shared between colours) and word-wide."""
import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from gpu_util import gpu_ctx, match_oracle

pytestmark = pytest.mark.gpu

RATES = dict(ka=1.0, kd=1.0, betaJ=0.4407)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


@pytest.mark.parametrize("model", ["ISING", "ADSDES"])
@pytest.mark.parametrize("q", [(8, 8), (16, 16), (32, 32), (16, 8)])
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_packed_matches_oracle(model, q, engine):
    lx, ly = 128, 64
    init = oracle.init_bernoulli(lx, ly, 33, 0.5)
    orc = oracle.FSRun(lx, ly, *q, model, RATES, init).run("STRANG", 0.1, 1.0, 8)
    with F.Context(lx, ly, model, RATES, q, bitpacked=True) as c:
        c.set_engine(engine)
        c.set_state(init)
        assert np.array_equal(c.get_state(), init)
        c.run("STRANG", 0.1, 1.0, 8)
        assert c.stats()["check_failures"] == 0
        match_oracle((c.get_state(), c.stats()["events"], c.workload()), orc,
                     lambda: gpu_ctx(lx, ly, q, model, RATES, init, engine=engine, packed=True),
                     lambda: oracle.FSRun(lx, ly, *q, model, RATES, init), "STRANG", 0.1, 1.0, 8,
                     what=f"packed {model} q={q} {engine}")
        cov, en, pc = c.observables(0, 8)
        ocov, oen, opc = oracle.observables(lx, ly, model, c.get_state(), 8)
        assert np.array_equal(cov, ocov) and en == oen and np.array_equal(pc, opc)


def test_packed_fp32_equals_unpacked_and_init():
    lx = ly = 256
    out = []
    for packed in (False, True):
        with F.Context(lx, ly, "ISING", RATES, (16, 16), bitpacked=packed) as c:
            c.set_clock("FP32")
            c.set_engine("PERSISTENT")
            c.init_random(5, 0.5)
            if packed:
                assert np.array_equal(c.get_state(), oracle.init_bernoulli(lx, ly, 5, 0.5))
            c.run("LIE", 0.5, 5.0, 5)
            out.append((c.get_state(), c.stats()["events"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]

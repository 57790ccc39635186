"""Processor communication schedules compared (Section 4.1): the weak error of
the Lie schedule shrinks with the cell size q (Eq. liebound: the commutator
lives on cell boundaries), while the random sub-lattice schedule's error is
O(1) in q (Eq. randomtimestep), so at equal tolerance Lie admits a much larger
window (Eq. pcscompare). Measured on 8,192-replica batches of 64x64
adsorption/desorption lattices (betaJ = 2) against a fine-window reference."""
import numpy as np
import pytest

import paper_1105_4673_gb300 as F

pytestmark = pytest.mark.gpu

L, NREP, T = 64, 8192, 2.0
RATES = dict(ka=1.0, kd=1.0, betaJ=2.0)


def _coverage(scheme, dt, q, seed):
    reps = [dict(lx=L, ly=L, rates=RATES)] * NREP
    with F.Context(model="ADSDES", q=(q, q), batch=reps) as b:
        b.set_clock("FP32")
        b.set_engine("PERSISTENT")
        b.init_random(seed, 0.5)
        b.run(scheme, dt, T, seed)
        return np.array([b.observables(r, 0)[0][1] for r in range(NREP)])


@pytest.fixture(scope="module")
def study():
    from paper_1105_4673_gb300 import build
    build.build()
    ref = _coverage("LIE", 1.0 / 64, 32, 4242)
    out = {}
    for q in (2, 8, 32):
        for scheme, dt in (("LIE", 1.0), ("RANDOM", 0.25)):
            c = _coverage(scheme, dt, q, 7000 + 37 * q + len(scheme))
            out[scheme, q] = (c.mean() - ref.mean(), np.sqrt(c.var() / NREP + ref.var() / NREP))
    return out


def test_random_schedule_error_is_order_one_in_q(study):
    b2, s2 = study["RANDOM", 2]
    b32, s32 = study["RANDOM", 32]
    assert abs(b2) > 10 * s2 and abs(b32) > 10 * s32
    assert abs(b2 - b32) < 4 * np.hypot(s2, s32)


def test_lie_error_shrinks_with_cell_size(study):
    b2, s2 = study["LIE", 2]
    b32, s32 = study["LIE", 32]
    assert abs(b2) > 5 * s2
    assert abs(b2) > abs(b32) + 3 * np.hypot(s2, s32)


def test_lie_allows_a_larger_window_at_equal_tolerance(study):
    for q in (2, 8, 32):
        assert abs(study["RANDOM", q][0]) > 5 * abs(study["LIE", q][0])

"""fskmc_observables_noalloc: the observables without any allocation.

Some callers cannot let a library allocate device memory (their memory
belongs to their own pool, or they read the state after running out of
memory). This entry point keeps its accumulators in a fixed device array
inside the library. Here it must give exactly what fskmc_observables gives
(the sums are exact integers, so the results are bit-identical), on two
calls in a row, since the array keeps the previous call's contents.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1105_4673_gb300 as F
from workloads import random_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _noalloc(ptr, lx, ly, model, rmax, stream):
    L = F.lib()
    cov = (C.c_double * 3)()
    en = C.c_double()
    pc = (C.c_double * max(2 * rmax, 1))()
    st = L.fskmc_observables_noalloc(ptr, lx, ly, F.MODELS[model], stream, cov, C.byref(en), pc,
                                     rmax)
    return st, np.array(cov[:]), en.value, np.array(pc[:2 * rmax])


@pytest.mark.parametrize("model,lx,ly,rmax1,rmax2", [("ISING", 128, 96, 32, 8),
                                                     ("ZGB", 64, 64, 16, 16)])
def test_noalloc_matches_observables_twice(model, lx, ly, rmax1, rmax2):
    import torch
    stream = torch.cuda.current_stream()
    nstates = 3 if model == "ZGB" else 2
    rates = dict(ka=1.0, kd=1.0, betaJ=0.5, yA=0.5, kr=2.0)
    with F.Context(lx, ly, model, rates, (8, 8), stream=stream) as c:
        for call, (seed, rmax) in enumerate([(1, rmax1), (2, rmax2)]):
            lat = random_lattice(lx, ly, nstates, seed)
            c.set_state(lat)
            want = c.observables(0, rmax)
            dev = torch.empty(lx * ly, dtype=torch.uint8, device="cuda")
            c.get_state(0, out=dev)
            c.sync()
            st, cov, en, pc = _noalloc(dev.data_ptr(), lx, ly, model, rmax, stream.cuda_stream)
            assert st == F.OK, f"call {call}"
            assert np.array_equal(cov, want[0]), f"call {call}"
            assert (np.isnan(en) and np.isnan(want[1])) or en == want[1], f"call {call}"
            assert np.array_equal(pc, want[2]), f"call {call}"


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    dev = torch.zeros(512 * 512, dtype=torch.uint8, device="cuda")
    st, *_ = _noalloc(dev.data_ptr(), 512, 512, "ISING", F.NOALLOC_MAX_RMAX + 1, None)
    assert st == F.EINVAL
    st, *_ = _noalloc(dev.data_ptr(), 512, 512, "ISING", F.NOALLOC_MAX_RMAX, None)
    assert st == F.OK
    st, *_ = _noalloc(None, 512, 512, "ISING", 4, None)
    assert st == F.EINVAL

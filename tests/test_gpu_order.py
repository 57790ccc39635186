"""Heaviest-first issue order (Section 6, Eq. wload): the order in which a
window's active cells are issued changes timing only. Lattices, event
counts and workloads are bit-identical under row-major and workload order,
in both engines, for in-place and ping-pong models and for batches."""
import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from gpu_util import gpu_ctx, match_oracle
from workloads import random_lattice

pytestmark = pytest.mark.gpu

RATES = {
    "ADSDES": dict(ka=1.0, kd=1.0, betaJ=1.0),
    "ISING": dict(ka=1.0, kd=1.0, betaJ=0.4407),
    "DIFFUSION": dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0),
    "ZGB": dict(yA=0.52, kr=100.0, kd=0.01),
    "ISING1D": dict(ka=1.0, kd=1.0, betaJ=2.0, betah=1.0),
}
GEOMS = {
    "ADSDES": (128, 96, (8, 8)),
    "ISING": (96, 64, (6, 8)),
    "DIFFUSION": (128, 128, (16, 16)),
    "ZGB": (192, 128, (16, 16)),
    "ISING1D": (8192, 1, (32, 1)),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _init(model, lx, ly, seed):
    if model == "ZGB":
        return random_lattice(lx, ly, 3, seed, p=[0.6, 0.2, 0.2])
    return oracle.init_bernoulli(lx, ly, seed, 0.3 if model == "DIFFUSION" else 0.5)


def _run(model, engine, order, scheme, steps=3):
    lx, ly, q = GEOMS[model]
    init = _init(model, lx, ly, 17)
    with F.Context(lx, ly, model, RATES[model], q) as c:
        c.set_engine(engine)
        c.set_task_order(order)
        c.set_state(init)
        # several runs so that later windows are ordered by real workloads
        for _ in range(steps):
            c.run(scheme, 0.05, 0.2, 4242)
        return c.get_state(), c.stats()["events"], c.workload()


@pytest.mark.parametrize("model", list(GEOMS))
@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
@pytest.mark.parametrize("scheme", ["LIE", "RANDOM"])
def test_workload_order_changes_nothing(model, engine, scheme):
    a = _run(model, engine, "NATURAL", scheme)
    b = _run(model, engine, "WORKLOAD", scheme)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
    assert a[1] > 0


@pytest.mark.parametrize("engine", ["PLAIN", "PERSISTENT"])
def test_workload_order_matches_oracle(engine):
    model, (lx, ly, q) = "DIFFUSION", GEOMS["DIFFUSION"]
    init = _init(model, lx, ly, 3)
    orc = oracle.FSRun(lx, ly, *q, model, RATES[model], init).run("RANDOM_ORDER", 0.05, 0.5, 99)
    with F.Context(lx, ly, model, RATES[model], q) as c:
        c.set_engine(engine)
        c.set_task_order("WORKLOAD")
        c.set_state(init)
        c.run("RANDOM_ORDER", 0.05, 0.25, 99)
        c.run("RANDOM_ORDER", 0.05, 0.25, 99)
        got = (c.get_state(), c.stats()["events"], c.workload())

    def make_gpu():
        g = gpu_ctx(lx, ly, q, model, RATES[model], init, engine=engine)
        g.set_task_order("WORKLOAD")
        return g
    match_oracle(got, orc, make_gpu, lambda: oracle.FSRun(lx, ly, *q, model, RATES[model], init),
                 "RANDOM_ORDER", 0.05, 0.5, 99, what=f"heaviest-first {engine}")


def test_workload_order_batch():
    reps = [dict(lx=s, ly=s, rates=dict(ka=1.0, kd=1.0, betaJ=b))
            for s, b in [(64, 0.3), (128, 0.9), (96, 0.5), (256, 0.2), (64, 1.5)]]
    out = {}
    for order in ("NATURAL", "WORKLOAD"):
        for engine in ("PLAIN", "PERSISTENT"):
            with F.Context(model="ADSDES", q=(8, 8), batch=reps) as b:
                b.set_engine(engine)
                b.set_task_order(order)
                b.init_random(5, 0.5)
                b.run("LIE", 0.1, 1.0, 7)
                b.run("LIE", 0.1, 1.0, 7)
                out[order, engine] = ([b.get_state(r) for r in range(len(reps))],
                                      b.stats()["events"])
    ref = out["NATURAL", "PLAIN"]
    for k, v in out.items():
        assert v[1] == ref[1], k
        assert all(np.array_equal(x, y) for x, y in zip(v[0], ref[0])), k


def test_task_order_rejects_unknown():
    with F.Context(64, 64, "ADSDES", RATES["ADSDES"], (8, 8)) as c:
        with pytest.raises(F.FskmcError):
            c.set_task_order(7)

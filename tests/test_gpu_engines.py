"""The persistent engine (one graph-launched kernel for every window of
every replica), batches of uneven replicas, the binary32 window clock and
the bounded-wait failure path."""
import numpy as np
import pytest

import oracle
import paper_1105_4673_gb300 as F
from gpu_util import gpu_ctx, match_oracle
from oracle import closed_forms as CF
from workloads import random_lattice

pytestmark = pytest.mark.gpu

RATES = {
    "ADSDES": dict(ka=1.0, kd=1.0, betaJ=1.0),
    "ISING": dict(ka=1.0, kd=1.0, betaJ=0.6),
    "DIFFUSION": dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0),
    "ZGB": dict(yA=0.52, kr=100.0, kd=0.01),
}


def _init(model, lx, ly, seed):
    if model == "ZGB":
        return random_lattice(lx, ly, 3, seed, p=[0.6, 0.2, 0.2])
    return oracle.init_bernoulli(lx, ly, seed, 0.3 if model == "DIFFUSION" else 0.5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


@pytest.mark.parametrize("model", list(RATES))
@pytest.mark.parametrize("scheme", ["LIE", "STRANG", "RANDOM"])
def test_persistent_fp64_matches_oracle(model, scheme):
    lx, ly, q = 64, 48, (8, 8)
    init = _init(model, lx, ly, 21)
    dt = 0.05
    orc = oracle.FSRun(lx, ly, *q, model, RATES[model], init).run(scheme, dt, 1.0, 99)
    with gpu_ctx(lx, ly, q, model, RATES[model], init, engine="PERSISTENT") as c:
        c.run(scheme, dt, 1.0, 99)
        st = c.stats()
        assert st["check_failures"] == 0 and st["timeouts"] == 0
        got = (c.get_state(), st["events"], c.workload())
    match_oracle(got, orc, lambda: gpu_ctx(lx, ly, q, model, RATES[model], init, engine="PERSISTENT"),
                 lambda: oracle.FSRun(lx, ly, *q, model, RATES[model], init), scheme, dt, 1.0, 99,
                 what=f"persistent {model} {scheme}")


def _batch():
    reps = [dict(lx=32, ly=32, rates=dict(ka=0.5, kd=1.0, betaJ=0.3)),
            dict(lx=64, ly=48, rates=dict(ka=2.0, kd=1.0, betaJ=0.8)),
            dict(lx=96, ly=64, rates=dict(ka=1.0, kd=1.0, betaJ=0.0)),
            dict(lx=16, ly=16, rates=dict(ka=0.1, kd=1.0, betaJ=0.5))]
    return reps


@pytest.mark.parametrize("scheme", ["LIE", "RANDOM_ORDER"])
def test_batch_replicas_match_single_contexts(scheme):
    reps = _batch()
    seed = 2024
    with F.Context(model="ADSDES", q=(8, 8), batch=reps) as b:
        b.init_random(seed, 0.5)
        b.set_engine("PERSISTENT")
        b.run(scheme, 0.1, 2.0, seed)
        assert b.stats()["check_failures"] == 0
        for r, rp in enumerate(reps):
            init = oracle.init_bernoulli(rp["lx"], rp["ly"], seed, 0.5, replica=r)
            orc = oracle.FSRun(rp["lx"], rp["ly"], 8, 8, "ADSDES", rp["rates"], init, replica=r)
            orc.run(scheme, 0.1, 2.0, seed)
            with gpu_ctx(rp["lx"], rp["ly"], (8, 8), "ADSDES", rp["rates"], init, replica=r) as s:
                s.run(scheme, 0.1, 2.0, seed)
                alone = (s.get_state(), s.stats()["events"], s.workload())
            got = b.get_state(r)
            assert np.array_equal(got, alone[0]), f"replica {r}: batch differs from single context"
            match_oracle(alone, orc,
                         lambda: gpu_ctx(rp["lx"], rp["ly"], (8, 8), "ADSDES", rp["rates"], init, replica=r),
                         lambda: oracle.FSRun(rp["lx"], rp["ly"], 8, 8, "ADSDES", rp["rates"], init, replica=r),
                         scheme, 0.1, 2.0, seed, replica=r, what=f"replica {r}")


@pytest.mark.parametrize("model", list(RATES))
def test_fp32_engines_agree_bitwise(model):
    """The binary32 clock is deterministic: plain and persistent engines and
    any launch shape give identical lattices."""
    lx, ly, q = 64, 64, (8, 8)
    init = _init(model, lx, ly, 5)
    out = []
    for engine, wpb in (("PLAIN", 4), ("PERSISTENT", 8), ("PLAIN", 1)):
        with gpu_ctx(lx, ly, q, model, RATES[model], init, clock="FP32", engine=engine, wpb=wpb) as c:
            c.run("STRANG", 0.05, 1.0, 17)
            out.append((c.get_state(), c.stats()["events"]))
    assert all(np.array_equal(out[0][0], o[0]) and out[0][1] == o[1] for o in out[1:])


def test_fp32_clock_noninteracting_closed_form():
    """betaJ = 0: every site is an independent two-state chain, so the
    coverage after T is the closed form whatever the schedule."""
    lx = ly = 256
    ka, kd, T = 2.0, 1.0, 1.0
    with F.Context(lx, ly, "ADSDES", dict(ka=ka, kd=kd, betaJ=0.0), (16, 16)) as c:
        c.set_clock("FP32")
        c.init_random(3, 0.5)
        th0 = c.get_state().mean()
        c.run("LIE", 0.05, T, 3)
        got = c.get_state().mean()
    want = CF.coverage_noninteracting(T, th0, ka, kd)
    assert abs(got - want) < 4 * np.sqrt(want * (1 - want) / (lx * ly))


@pytest.mark.parametrize("model", ["ADSDES", "ZGB"])
def test_fp32_and_fp64_clocks_agree_statistically(model):
    """Observables of the binary32-clock form agree with the binary64 form
    within 3 standard errors over independent replicas."""
    n, L = 64, 64
    reps = [dict(lx=L, ly=L, rates=RATES[model]) for _ in range(n)]
    means = {}
    for clock in ("FP64", "FP32"):
        with F.Context(model=model, q=(8, 8), batch=reps) as b:
            b.set_clock(clock)
            b.set_engine("PERSISTENT")
            b.init_random(77 if clock == "FP64" else 78, 0.5 if model != "ZGB" else 0.0)
            b.run("LIE", 0.1, 2.0, 11 if clock == "FP64" else 12)
            means[clock] = np.array([b.observables(r, 1)[0][1] for r in range(n)])
    d = means["FP32"].mean() - means["FP64"].mean()
    se = np.sqrt(means["FP32"].var(ddof=1) / n + means["FP64"].var(ddof=1) / n)
    assert abs(d) < 3 * se + 1e-12, (d, se)


def test_diffusion_conserves_particles_on_gpu():
    lx = ly = 64
    init = oracle.init_bernoulli(lx, ly, 8, 0.3)
    for engine in ("PLAIN", "PERSISTENT"):
        with gpu_ctx(lx, ly, (8, 8), "DIFFUSION", dict(ka=0.0, kd=0.0, betaJ=1.0, nu=10.0), init,
                     engine=engine) as c:
            c.run("RANDOM", 0.05, 1.0, 6)
            got = c.get_state()
            assert c.stats()["events"] > 10000
            assert int(got.sum()) == int(init.sum())


def test_bounded_wait_gives_up_cleanly():
    """A persistent run whose waits are limited to zero polls must give up
    with ETIMEOUT (no hang, no fault), and the context stays usable."""
    lx = ly = 256
    with F.Context(lx, ly, "ISING", RATES["ISING"], (8, 8)) as c:
        c.set_engine("PERSISTENT")
        c.init_random(1, 0.5)
        c.set_spin_limit(0)
        with pytest.raises(F.FskmcError) as e:
            c.run("LIE", 0.5, 20.0, 1)
        assert e.value.status == F.ETIMEOUT
        assert c.stats()["timeouts"] >= 1
        c.set_spin_limit(1 << 24)
        c.init_random(1, 0.5)
        c.run("LIE", 0.5, 2.0, 1)
        assert c.stats()["check_failures"] == 0


def test_autotuner_picks_a_valid_shape():
    reps = _batch()
    q, wpb, rate = F.autotune(reps, "ADSDES", "LIE", 0.1, clock="FP32", engine="PERSISTENT")
    assert q[0] == q[1] and q[0] in (8, 16) and wpb in (2, 4, 8) and rate > 0
    with F.Context(model="ADSDES", q=q, batch=reps) as b:
        b.set_warps_per_block(wpb)
        b.set_engine("PERSISTENT")
        b.init_random(1, 0.5)
        b.run("LIE", 0.1, 1.0, 1)
        assert b.stats()["check_failures"] == 0


def test_integer_divide_matches_hardware():
    """The binary64 waiting time divides on the integer pipes; it must agree
    bit for bit with the hardware correctly rounded divide, including exact
    quotients, zero numerators, and quotients outside the normal range
    (handled by the fallback)."""
    rng = np.random.default_rng(7)
    n = 1 << 21
    a = 40.0 * rng.random(n)
    a[::5] *= 1e-10
    a[::97] = 0.0
    b = 1e-6 * np.exp(32.0 * rng.random(n))
    b[::101] = 1.0
    b[::103] = 3.0
    a[::103] = 3.0 * np.arange(len(a[::103]))
    # extreme ratios: results beyond the normal range use the fallback
    a[1:200] = 1e300
    b[1:200] = 1e-300
    a[200:400] = 1e-300
    b[200:400] = 1e300
    # significands straddling: a's below and above b's
    a[400:600] = np.nextafter(b[400:600], 0)
    a[600:800] = np.nextafter(b[600:800], np.inf)
    assert F.selftest_divide(a, b) == 0


def test_device_log_matches_host_log():
    """The window clock's table-driven binary64 -log(u_t), u_t = n 2^-53, agrees
    with the host logarithm to one unit in the last place and equals it for
    almost every draw; u_t = 1 gives 0."""
    rng = np.random.default_rng(11)
    n = rng.integers(1, 2 ** 53, size=1 << 20, dtype=np.uint64, endpoint=True)
    edges = np.array([1, 2, 3, 2 ** 52, 2 ** 52 + 1, 3 * 2 ** 51 - 1, 3 * 2 ** 51, 2 ** 53 - 1, 2 ** 53],
                     dtype=np.uint64)
    n = np.concatenate([edges, n, (2 ** 53 - rng.integers(0, 2 ** 20, size=4096)).astype(np.uint64)])
    got = F.selftest_log(n)
    ref = -np.log(n.astype(np.float64) * 2.0 ** -53)
    assert got[8] == 0.0 and ref[8] == 0.0
    nz = ref != 0
    ulps = np.abs(got[nz] - ref[nz]) / np.spacing(np.abs(ref[nz]))
    assert ulps.max() <= 1.0, ulps.max()
    assert (got == ref).mean() > 0.99

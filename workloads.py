"""Seeded synthetic workloads shaped like the paper's benchmarks.

Shared by the tests, the benchmark and the smoke check. It holds only
workload descriptions and seeded parameter draws (numpy), none of the
method's arithmetic: initial lattices are drawn by each implementation
from the counter-based generator keyed by the seed given here.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x5EED0000

# The six workloads. Sizes, rates and schedules follow the paper's test
# problems: non-interacting and interacting adsorption/desorption (Section 4.1),
# the 2D Ising benchmark (Section 7), adsorption/desorption with surface
# diffusion (Section 2), an ensemble of replicas (Section 7's M independent
# realisations), the ZGB catalysis model (Section 7.1) and the 1D Ising ring
# (Section 7).
WORKLOADS = {
    "adsdes64": dict(lx=64, ly=64, model="ADSDES", rates=dict(ka=1.0, kd=1.0, betaJ=1.0),
                     q=(8, 8), scheme="LIE", dt=0.1, T=10.0, coverage=0.5,
                     seed=SEED_BASE + 0),
    "ising1024": dict(lx=1024, ly=1024, model="ISING",
                      rates=dict(ka=1.0, kd=1.0, betaJ=0.4407), q=(16, 16), scheme="LIE",
                      dt=1.0, T=1000.0, coverage=0.5, bitpacked=True, seed=SEED_BASE + 1),
    "diffusion4096": dict(lx=4096, ly=4096, model="DIFFUSION",
                          rates=dict(ka=1.0, kd=1.0, betaJ=2.0, nu=10.0), q=(32, 32),
                          scheme="RANDOM_ORDER", dt=0.05, T=100.0, coverage=0.3,
                          seed=SEED_BASE + 2),
    "ensemble512": dict(n=512, model="ADSDES", scheme="LIE", dt=0.1, T=50.0, coverage=0.5,
                        seed=SEED_BASE + 3),
    "zgb16384": dict(lx=16384, ly=16384, model="ZGB",
                     rates=dict(yA=0.52, kr=100.0, kd=0.01), q=(32, 32), scheme="STRANG",
                     dt=0.02, T=200.0, bump=dict(amp=0.9, width=16384 / 8), seed=SEED_BASE + 4),
    # the 1D Ising benchmark of Section 7: a ring of N = 2^15 sites, K = 1,
    # beta = 4, h = 1 (betaJ = beta K, betah = beta h), dt = 1.0
    "ising1d32768": dict(lx=32768, ly=1, model="ISING1D",
                         rates=dict(ka=1.0, kd=1.0, betaJ=4.0, betah=4.0), q=(32, 1),
                         scheme="LIE", dt=1.0, T=1000.0, coverage=0.5, bitpacked=True,
                         seed=SEED_BASE + 5),
}


def cpu_sample(w: dict, threads: int = 1) -> tuple[int, int]:
    """A bounded sample of a workload for the host-CPU oracle timing: a
    256 x 256 lattice (a ring of 8192 sites for the 1D model) for one
    thread; for the all-core form a lattice with at least 16 active cells
    per thread (up to 2048 x 2048), so that every thread has cells to run."""
    if w["model"] == "ISING1D":
        n = 8192
        while threads > 1 and n // w["q"][0] // 2 < 16 * threads and n < (1 << 20):
            n *= 2
        return n, 1
    side = 256
    qx, qy = w["q"]
    while threads > 1 and (side // qx) * (side // qy) // 2 < 16 * threads and side < 2048:
        side *= 2
    return side, side


def ensemble_replicas(n: int = 512, seed: int = SEED_BASE + 3):
    """Per-replica (side, rates) of the batched ensemble: sides uniform on
    {64, 128, 256, 512}, betaJ uniform on [0.2, 0.8], ka/kd log-uniform on
    [0.1, 10] with kd = 1."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([64, 128, 256, 512], size=n)
    betaJ = rng.uniform(0.2, 0.8, size=n)
    ratio = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=n))
    return [dict(lx=int(s), ly=int(s), rates=dict(ka=float(r), kd=1.0, betaJ=float(b)))
            for s, b, r in zip(sides, betaJ, ratio)]


def random_lattice(lx: int, ly: int, nstates: int, seed: int, p=None) -> np.ndarray:
    """A seeded random lattice (uint8, row-major) for parity cases: state s
    with probability p[s] (uniform if None), probabilities rounded to
    multiples of 1/256 so that full-size lattices need no wide temporaries."""
    rng = np.random.default_rng(seed)
    p = np.full(nstates, 1.0 / nstates) if p is None else np.asarray(p, float)
    cut = np.round(np.cumsum(p) * 256).astype(np.int64)[:-1]
    u = rng.integers(0, 256, size=lx * ly, dtype=np.uint8)
    out = np.zeros(lx * ly, np.uint8)
    for c in cut:
        out += (u >= c).astype(np.uint8)
    return out

"""The seeded synthetic workloads keep the shapes of the paper's test
problems (Sections 2, 4.1, 7 and 7.1): lattice sizes and cells that admit
the checkerboard, the stated rates and schedules, and the batched ensemble's
recipe -- sides uniform on {64, 128, 256, 512}, betaJ uniform on
[0.2, 0.8], k_a/k_d log-uniform on [0.1, 10] -- drawn reproducibly from its
seed."""
import numpy as np

from workloads import WORKLOADS, cpu_sample, ensemble_replicas


def test_lattices_admit_the_checkerboard():
    for name, w in WORKLOADS.items():
        if "lx" not in w:
            continue
        qx, qy = w["q"]
        assert w["lx"] % (2 * qx) == 0, name
        if w["ly"] > 1:
            assert w["ly"] % (2 * qy) == 0, name
        # whole windows over the run
        assert abs(round(w["T"] / w["dt"]) - w["T"] / w["dt"]) < 1e-9, name


def test_stated_shapes_and_rates():
    assert (WORKLOADS["ising1024"]["lx"], WORKLOADS["ising1024"]["q"]) == (1024, (16, 16))
    assert WORKLOADS["ising1024"]["rates"]["betaJ"] == 0.4407  # near the critical coupling
    assert WORKLOADS["ising1024"]["bitpacked"]
    assert WORKLOADS["diffusion4096"]["scheme"] == "RANDOM_ORDER"
    assert WORKLOADS["zgb16384"]["scheme"] == "STRANG" and WORKLOADS["zgb16384"]["q"] == (32, 32)
    assert WORKLOADS["ising1d32768"]["ly"] == 1 and WORKLOADS["ising1d32768"]["lx"] == 1 << 15
    assert cpu_sample(WORKLOADS["ising1d32768"]) == (8192, 1)
    assert cpu_sample(WORKLOADS["ising1024"]) == (256, 256)
    # the all-core sample gives every thread at least 16 active cells
    for name in ("zgb16384", "ising1024", "diffusion4096", "ising1d32768"):
        w = WORKLOADS[name]
        lx, ly = cpu_sample(w, 16)
        assert (lx // w["q"][0]) * (ly // w["q"][1]) // 2 >= 16 * 16, name


def test_ensemble_recipe():
    reps = ensemble_replicas()
    assert len(reps) == 512
    assert reps == ensemble_replicas()  # seeded
    sides = np.array([r["lx"] for r in reps])
    assert set(sides) <= {64, 128, 256, 512} and len(set(sides)) == 4
    assert all(r["lx"] == r["ly"] for r in reps)
    b = np.array([r["rates"]["betaJ"] for r in reps])
    assert b.min() >= 0.2 and b.max() <= 0.8
    ratio = np.array([r["rates"]["ka"] / r["rates"]["kd"] for r in reps])
    assert ratio.min() >= 0.1 and ratio.max() <= 10.0
    lr = np.log10(ratio)
    # log-uniform on [-1, 1]: mean 0, variance 1/3 (512 draws: well within 4 standard errors)
    assert abs(lr.mean()) < 4 * np.sqrt(1 / 3 / 512)
    assert abs(lr.var() - 1 / 3) < 0.1
    # every side occurs about a quarter of the time
    for s in (64, 128, 256, 512):
        assert abs((sides == s).mean() - 0.25) < 0.08

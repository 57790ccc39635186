"""Whole-batch state transfer: fskmc_state_layout, fskmc_set_state_all and
fskmc_get_state_all move every replica of a batch (Section 7's independent
realisations) in one copy each way. They must agree byte for byte with the
per-replica calls, from host and from device buffers, refuse a byte that is
not a state of the model (leaving every lattice cleared), and refuse a
bit-packed context."""
import numpy as np
import pytest

import paper_1105_4673_gb300 as F
from workloads import random_lattice

pytestmark = pytest.mark.gpu

RATES = {
    "ADSDES": [dict(ka=1.0, kd=1.0, betaJ=1.0), dict(ka=0.5, kd=2.0, betaJ=0.3), dict(ka=2.0, kd=0.2, betaJ=0.8)],
    "ZGB": [dict(yA=0.52, kr=10.0, kd=0.1), dict(yA=0.4, kr=1.0, kd=0.0), dict(yA=0.6, kr=5.0, kd=0.5)],
    "DIFFUSION": [dict(ka=1.0, kd=1.0, betaJ=1.0, nu=10.0)] * 3,
}
SIZES = [(64, 64), (96, 32), (32, 160)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1105_4673_gb300 import build
    build.build()


@pytest.mark.parametrize("model", ["ADSDES", "ZGB", "DIFFUSION"])
def test_state_all_matches_per_replica_calls(model):
    import torch
    nst = 3 if model == "ZGB" else 2
    reps = [dict(lx=lx, ly=ly, rates=r) for (lx, ly), r in zip(SIZES, RATES[model])]
    with F.Context(model=model, q=(8, 8), batch=reps) as b:
        lay = b.state_layout()
        assert lay[0] == 0 and np.all(lay[:-1] % 256 == 0)
        for r, (lx, ly) in enumerate(SIZES):
            assert lay[r + 1] >= lay[r] + lx * ly
        total = int(lay[-1])
        lats = [random_lattice(lx, ly, nst, 31 + r) for r, (lx, ly) in enumerate(SIZES)]
        buf = np.zeros(total, np.uint8)
        for r, g in enumerate(lats):
            buf[lay[r]:lay[r] + g.size] = g
        b.set_state_all(buf)
        for r, g in enumerate(lats):
            assert np.array_equal(b.get_state(r), g)
        b.run("LIE", 0.1, 0.5, 3)
        out = b.get_state_all()
        assert out.size == total
        for r, (lx, ly) in enumerate(SIZES):
            assert np.array_equal(out[lay[r]:lay[r] + lx * ly], b.get_state(r))
        # device buffers: the same bytes both ways
        dbuf = torch.from_numpy(out.copy()).cuda()
        b.set_state_all(dbuf)
        dout = torch.empty(total, dtype=torch.uint8, device="cuda")
        b.get_state_all(dout)
        torch.cuda.synchronize()
        assert np.array_equal(dout.cpu().numpy(), out)
        # a byte that is not a state of the model: refused, every lattice cleared
        bad = out.copy()
        bad[lay[1] + 5] = 7
        with pytest.raises(F.FskmcError):
            b.set_state_all(bad)
        assert not b.get_state_all().any()


def test_state_all_refuses_bitpacked_context():
    with F.Context(64, 64, "ISING", dict(ka=1.0, kd=1.0, betaJ=0.4), (16, 16), bitpacked=True) as c:
        with pytest.raises(F.FskmcError):
            c.set_state_all(np.zeros(64 * 64, np.uint8))
        with pytest.raises(F.FskmcError):
            c.get_state_all(np.zeros(64 * 64, np.uint8))

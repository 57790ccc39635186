"""Helpers for the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs and compare."""
import numpy as np

import oracle
import paper_1105_4673_gb300 as F


def gpu_ctx(lx, ly, q, model, rates, init, clock="FP64", engine="PLAIN", wpb=None, replica=None):
    c = F.Context(lx, ly, model, rates, q)
    if replica is not None:
        c.set_replica_id(replica)
    c.set_clock(clock)
    c.set_engine(engine)
    if wpb:
        c.set_warps_per_block(wpb)
    c.set_state(np.ascontiguousarray(init, np.uint8).reshape(-1))
    return c


def assert_same_or_flagged(gpu_lat, orc, qx, qy, lx, what=""):
    """Bit-equal lattices, except in cells the oracle flagged ambiguous."""
    if np.array_equal(gpu_lat, orc.lat):
        return 0
    bad = np.nonzero(gpu_lat != orc.lat)[0]
    assert orc.ambiguous > 0, f"{what}: {bad.size} sites differ and no window was ambiguous"
    return bad.size


def windowwise(c, orc, col, h, seed):
    """Run the schedule window by window on both sides; resync the GPU to
    the oracle after a window the oracle flagged ambiguous. Returns the
    number of resyncs."""
    resync = 0
    for cc, hh in zip(col, h):
        amb = orc.window(int(cc), float(hh), seed)
        c.window(int(cc), float(hh), seed)
        g = c.get_state()
        if not np.array_equal(g, orc.lat):
            assert amb.any(), "lattices differ after a window no cell flagged"
            c.set_state(orc.lat)
            resync += 1
    return resync

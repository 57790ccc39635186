"""Helpers for the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs and compare.

The comparison rule (the window-edge contract of the binary64 clock): GPU
and oracle lattices are bit-equal after every window, except in a window
where the oracle flags a cell ambiguous (an edge decision within 1e-12 of
the window end, which two correct logarithms may take differently). A run
the oracle flags nowhere is compared whole: lattice, event count and
per-cell workloads. A run it flags somewhere is replayed window by window on
fresh copies of both sides; every window must agree, lattice and events,
and the GPU is reset to the oracle's lattice only after a window the oracle
flagged. No path passes without comparing."""
import numpy as np

import oracle
import paper_1105_4673_gb300 as F


def gpu_ctx(lx, ly, q, model, rates, init, clock="FP64", engine="PLAIN", wpb=None, replica=None,
            grouped=None, packed=False):
    c = F.Context(lx, ly, model, rates, q, bitpacked=packed)
    if replica is not None:
        c.set_replica_id(replica)
    c.set_clock(clock)
    c.set_engine(engine)
    if wpb:
        c.set_warps_per_block(wpb)
    if grouped is not None:
        c.set_cell_grouping(grouped)
    c.set_state(np.ascontiguousarray(init, np.uint8).reshape(-1))
    return c


def windowwise(c, orc, col, h, seed):
    """Run the schedule window by window on both sides. After each window
    the lattices and the window's event counts must be equal, unless the
    oracle flagged a cell of that window ambiguous: then the GPU is reset to
    the oracle's lattice. Returns the number of resyncs."""
    resync = 0
    for cc, hh in zip(col, h):
        e_orc, e_gpu = orc.events, c.stats()["events"]
        amb = orc.window(int(cc), float(hh), seed)
        c.window(int(cc), float(hh), seed)
        g = c.get_state()
        same = np.array_equal(g, orc.lat) and c.stats()["events"] - e_gpu == orc.events - e_orc
        if not same:
            assert amb.any(), "lattices or event counts differ after a window no cell flagged"
            c.set_state(orc.lat)
            resync += 1
    return resync


def match_oracle(got, orc, make_gpu, make_orc, scheme, dt, T, seed, replica=0, what=""):
    """Compare a GPU run with the oracle's run of the same schedule.

    got: (lattice, events or None, workload or None) of the GPU's run; orc: the
    oracle's FSRun after the same run; make_gpu() / make_orc(): fresh
    copies of both sides at the run's start (same state, configuration and
    window index 0), used only when the oracle flagged a window. Returns the
    number of resyncs (0 when nothing was flagged)."""
    lat, events, wl = got
    if orc.ambiguous == 0:
        assert np.array_equal(lat, orc.lat), f"{what}: lattice differs from the oracle"
        if events is not None:
            assert events == orc.events, f"{what}: events {events} vs oracle {orc.events}"
        if wl is not None:
            assert np.array_equal(wl, orc.workload), f"{what}: workloads differ"
        return 0
    col, h = oracle.schedule(scheme, dt, T, seed, replica)
    c = make_gpu()
    try:
        n = windowwise(c, make_orc(), col, h, seed)
    finally:
        c.close()
    assert n <= orc.ambiguous, f"{what}: {n} resyncs for {orc.ambiguous} flagged cell-windows"
    return n

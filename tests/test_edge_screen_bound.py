"""The screened window-edge check of the binary64 clock, emulated on the CPU.

The kernels decide whether an event's end, fl(tau + fl(l / lambda)) in
binary64 (Eq. skeleton), lies before the window length h from a binary32
estimate of the waiting time on an exact 64-bit integer clock in units of
h 2^-62 with a running error bound, and leave the events the estimate cannot
decide to the binary64 clock. This test replays long event sequences in exact
binary64 (Python floats: correctly rounded division and addition) beside an
emulation of the estimate -- l rounded toward zero, lambda truncated to
binary32, the reciprocal taken one unit in the last place low or high
(the approximate reciprocal's worst case, in whichever direction makes a
wrong decision likelier), binary32 products rounded to nearest -- and checks
that every decision the estimate takes is the binary64 one, including
windows built to end just inside and just outside the bound.
"""
import math
import random

import numpy as np

TWO62 = 1 << 62


def f32_bits(x):
    return int(np.array([x], np.float32).view(np.uint32)[0])


def bits_f32(b):
    return np.array([b], np.uint32).view(np.float32)[0]


def f64_bits(x):
    return int(np.array([x], np.float64).view(np.uint64)[0])


def f32_rz(x):
    """x (binary64, positive) rounded toward zero to binary32."""
    f = np.float32(x)
    if float(f) > x:
        f = np.nextafter(f, np.float32(0))
    return f


def screen(l, lam, sf, clk, err, near, rcp_dir):
    """The estimate Q, its bound E and the decision (take, unsure), as the
    kernels form them; rcp_dir = -1 / 0 / +1 moves the reciprocal one unit
    in the last place down, not at all, or up."""
    lb = f64_bits(lam)
    fe = (lb >> 52) - 896
    inrange = 1 <= fe <= 250
    lamf = bits_f32(((fe & 0xFF) << 23) | ((lb >> 29) & 0x7FFFFF)) if inrange else np.float32(1)
    rr = np.float32(1) / lamf
    if rcp_dir < 0:
        rr = np.nextafter(rr, np.float32(0))
    elif rcp_dir > 0:
        rr = np.nextafter(rr, np.float32(np.inf))
    lf = f32_rz(l)
    with np.errstate(over="ignore"):
        qf = np.float32(np.float32(lf * rr) * sf)
    qb = f32_bits(qf)
    qe = (qb >> 23) - 150
    qm = (qb & 0x7FFFFF) | 0x800000
    if qe >= 40:
        Q = 1 << 63
    elif qe >= 0:
        Q = qm << qe
    elif qe > -24:
        Q = qm >> -qe
    else:
        Q = 0
    E = err + (Q >> 20) + 2048
    rem = TWO62 - clk
    take = inrange and Q + E < rem
    unsure = near or (not inrange) or (not take and Q < rem + E)
    return Q, E, take, unsure


def run_window(rng, h, lams, rcp_dir, max_events=100000):
    """One window: events until the binary64 end passes h. Returns the
    number of screened decisions and of binary64 ones."""
    sf = np.float32(2.0 ** 62 / h)
    tau, clk, err, near = 0.0, 0, 0, False
    decided = exact = 0
    for _ in range(max_events):
        lam = lams(rng)
        n = rng.getrandbits(53) + 1                    # u_t = n 2^-53 in (0, 1]
        l = -math.log(n * 2.0 ** -53)
        end = tau + l / lam                            # binary64: fl(tau + fl(l / lam))
        take_exact = end < h
        Q, E, take, unsure = screen(l, lam, sf, clk, err, near, rcp_dir)
        if unsure:
            exact += 1
            take = take_exact
            near = True
        else:
            decided += 1
            assert take == take_exact, (tau, l, lam, h, Q, E, clk)
        if not take:
            break
        clk += Q
        err = E
        tau = end
    return decided, exact


def test_screen_never_contradicts_binary64():
    rng = random.Random(20261204)
    total_decided = total_exact = 0
    windows = 0
    for trial in range(120):
        h = 10.0 ** rng.uniform(-3, 3)
        scale = 10.0 ** rng.uniform(-2, 3) / h         # 0.01 .. 1000 events per window on average
        spread = rng.choice([1.0, 4.0, 100.0])
        lams = lambda r, s=scale, sp=spread: s * sp ** r.uniform(-1, 1)
        for rcp_dir in (-1, 0, 1):
            d, x = run_window(rng, h, lams, rcp_dir)
            total_decided += d
            total_exact += x
            windows += 1
    assert total_decided > 10000
    # the estimate decides nearly everything: about one binary64 decision per
    # window that ends near its edge, plus the rest of that window
    assert total_exact < 0.02 * total_decided + 4 * windows


def test_screen_at_the_bound():
    """Windows whose binary64 end of some event lies a hair inside or
    outside h, at distances around the screen's bound (2^-20 of h): the
    estimate must either decide correctly or leave it to binary64."""
    rng = random.Random(7)
    for trial in range(3000):
        lam = 10.0 ** rng.uniform(-1, 3)
        # a few events to build up the clock, then one that ends near h
        ls = [-math.log((rng.getrandbits(53) + 1) * 2.0 ** -53) for _ in range(rng.randint(0, 40))]
        tau = 0.0
        for l in ls:
            tau = tau + l / lam
        l_last = -math.log((rng.getrandbits(53) + 1) * 2.0 ** -53)
        end = tau + l_last / lam
        rel = rng.choice([-1, 1]) * 2.0 ** -rng.uniform(16, 30)
        h = end * (1.0 + rel)
        if not h > tau:
            continue
        sf = np.float32(2.0 ** 62 / h)
        for rcp_dir in (-1, 0, 1):
            clk, err, near, t = 0, 0, False, 0.0
            ok = True
            for l in ls + [l_last]:
                e_end = t + l / lam
                take_exact = e_end < h
                Q, E, take, unsure = screen(l, lam, sf, clk, err, near, rcp_dir)
                if unsure:
                    take, near = take_exact, True
                else:
                    assert take == take_exact, (trial, rcp_dir, rel, Q, E, clk)
                if not take:
                    ok = False
                    break
                clk, err, t = clk + Q, E, e_end
            assert ok == (end < h)


def test_screen_refuses_waits_beyond_the_window():
    """A waiting time far past the window (a nearly empty cell) is refused
    by the estimate alone, including one beyond the binary32 range of the
    integer clock."""
    sf = np.float32(2.0 ** 62 / 1.0)
    for lam in (1e-30, 1e-6, 0.5):
        Q, E, take, unsure = screen(30.0, lam, sf, 0, 0, False, 0)
        assert not take and not unsure

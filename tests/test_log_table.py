"""The binary64 logarithm of the window clock (-log(u_t), u_t = n 2^-53):
its table (generated by paper_1105_4673_gb300/csrc/gen_logtab.py) and the
reduction it relies on, checked on the CPU in exact rational arithmetic
against a 50-digit logarithm. The device's values are compared with numpy's
logarithm in tests/test_gpu_engines.py."""
import decimal
import importlib.util
import math
import os
import random
import struct
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1105_4673_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_logtab", os.path.join(CSRC, "gen_logtab.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_header_is_the_generator_output(gen, tmp_path, monkeypatch):
    monkeypatch.setattr(gen, "HERE", str(tmp_path))
    gen.main()
    assert (tmp_path / "fskmc_logtab.h").read_text() == open(os.path.join(CSRC, "fskmc_logtab.h")).read()


def test_table_entries(gen):
    decimal.getcontext().prec = 60
    rows = gen.table()
    assert len(rows) == 128
    for i, (invc, hi, lo) in enumerate(rows):
        f = Fraction(invc)
        scaled = f * (256 if f < 1 else 128)
        assert f == 1 or (scaled.denominator == 1 and scaled < 256), i  # 8 significant bits
        assert (Fraction(hi) * 2 ** 42).denominator == 1, i            # hi on the 2^-42 grid
        exact = -(decimal.Decimal(f.numerator) / decimal.Decimal(f.denominator)).ln()
        assert abs(decimal.Decimal(hi) + decimal.Decimal(lo) - exact) < decimal.Decimal(2) ** -95, i
    assert rows[0][0] == 1.0 and rows[127][0] == 1.0                   # no cancellation next to 1
    l2h, l2l = gen.ln2_parts()
    assert (Fraction(l2h) * 2 ** 42).denominator == 1
    assert abs(decimal.Decimal(l2h) + decimal.Decimal(l2l) - decimal.Decimal(2).ln()) < decimal.Decimal(2) ** -95


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _neg_log(n, rows, l2h, l2l):
    """The device algorithm, step for step, with exactly rounded binary64
    operations."""
    lz = 64 - n.bit_length()
    frac = (((n << lz) << 1) & (2 ** 64 - 1)) >> 12
    i = frac >> 45
    half = i >= 64
    m = struct.unpack("<d", struct.pack("<Q", ((1022 if half else 1023) << 52) | frac))[0]
    me = lz - 10 - (1 if half else 0)
    invc, lch, lcl = rows[i]
    r = _fma(m, invc, -1.0)
    assert Fraction(r) == Fraction(m) * Fraction(invc) - 1          # the reduction is exact
    q = _fma(r, -0.125, 1.0 / 7.0)
    for c in (-1.0 / 6.0, 0.2, -0.25, 1.0 / 3.0, -0.5):
        q = _fma(r, q, c)
    r2 = float(Fraction(r) * Fraction(r))
    hi = _fma(-float(me), l2h, lch)
    assert Fraction(hi) == -me * Fraction(l2h) + Fraction(lch)      # exact by construction
    lo = _fma(-float(me), l2l, lcl)
    tail = float(Fraction(r) + Fraction(_fma(r2, q, lo)))
    return float(0 - (Fraction(hi) + Fraction(tail)))


def test_logarithm_within_two_thirds_ulp(gen):
    decimal.getcontext().prec = 50
    rows = gen.table()
    l2h, l2l = gen.ln2_parts()
    rnd = random.Random(5)
    ns = [1, 2, 3, 2 ** 52, 2 ** 52 + 1, 3 * 2 ** 51 - 1, 3 * 2 ** 51, 2 ** 53 - 1, 2 ** 53]
    ns += [rnd.getrandbits(53) + 1 for _ in range(1500)]
    ns += [2 ** 53 - rnd.getrandbits(25) for _ in range(300)]        # u just below 1
    ns += [3 * 2 ** 51 + rnd.getrandbits(20) - 2 ** 19 for _ in range(300)]  # the m = 1.5 seam
    worst = 0.0
    for n in ns:
        got = _neg_log(n, rows, l2h, l2l)
        ex = -(decimal.Decimal(n) / decimal.Decimal(2 ** 53)).ln()
        if ex == 0:
            assert got == 0.0
            continue
        err = abs(float((decimal.Decimal(got) - ex) / decimal.Decimal(math.ulp(float(ex)))))
        worst = max(worst, err)
    assert worst < 0.67, worst

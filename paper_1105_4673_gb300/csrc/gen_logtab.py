"""Write fskmc_logtab.h: the tables of the binary64 logarithm used by the
window kernels for the waiting-time numerator -log(u_t).

The method is the table-driven reduction of P. T. P. Tang, "Table-driven
implementation of the logarithm function in IEEE floating-point arithmetic",
ACM TOMS 16 (1990), in its reciprocal-table form: for m in [0.75, 1.5) and
a table point c near m with a short reciprocal invc (8 significant bits),

    log(m) = -log(invc) + log1p(r),   r = m * invc - 1,

where r is exact in binary64 (one fused multiply-add: the product of a
53-bit and an 8-bit significand minus 1 fits in 53 bits because |r| < 2^-7)
and log1p(r) is a short polynomial. -log(invc) is stored as hi + lo with hi
a multiple of 2^-42, so that e*ln2_hi + hi is exact for |e| < 2^11.

Entries: index i = the top 7 fraction bits of m in [1, 2); i < 64 covers
m in [1 + i/128, 1 + (i+1)/128); i >= 64 covers m/2 in [0.5 + i/256,
0.5 + (i+1)/256) (the reduction uses m/2 there so that m in [0.75, 1.5)).
The two entries next to 1 (i = 0 and i = 127) use invc = 1 exactly, so that
r = m - 1 and no cancellation occurs near log(1) = 0.

Run: python gen_logtab.py  (rewrites fskmc_logtab.h beside this file).
"""
from __future__ import annotations

import decimal
import os
from fractions import Fraction

D = decimal.Decimal
decimal.getcontext().prec = 60
HERE = os.path.dirname(os.path.abspath(__file__))
Q = Fraction(1, 2 ** 42)


def table():
    rows = []
    for i in range(128):
        if i in (0, 127):
            invc = Fraction(1)
            lo_m, hi_m = ((Fraction(1), Fraction(1) + Fraction(1, 128)) if i == 0 else
                          (Fraction(1, 2) + Fraction(127, 256), Fraction(1)))
        elif i < 64:
            lo_m = Fraction(1) + Fraction(i, 128)
            hi_m = lo_m + Fraction(1, 128)
            c = (lo_m + hi_m) / 2
            invc = Fraction(round(Fraction(256) / c), 256)  # 8 significant bits, in (0.5, 1)
        else:
            lo_m = Fraction(1, 2) + Fraction(i, 256)
            hi_m = lo_m + Fraction(1, 256)
            c = (lo_m + hi_m) / 2
            invc = Fraction(round(Fraction(128) / c), 128)  # 8 significant bits, in (1, 2)
        scaled = invc * (256 if invc < 1 else 128)  # 8 significant bits: an integer below 256
        assert scaled.denominator == 1 and scaled < 256 or invc == 1, (i, invc)
        r_max = max(abs(lo_m * invc - 1), abs(hi_m * invc - 1))
        assert r_max <= Fraction(1, 128), (i, float(r_max))  # hi_m itself is excluded
        logc = -(D(invc.numerator) / D(invc.denominator)).ln()
        hi = Fraction(round(Fraction(logc) / Q)) * Q
        lo = float(Fraction(logc) - hi)
        assert float(hi) == hi
        rows.append((float(invc), float(hi), lo))
    return rows


def ln2_parts():
    ln2 = D(2).ln()
    hi = Fraction(round(Fraction(ln2) / Q)) * Q
    return float(hi), float(Fraction(ln2) - hi)


def main():
    rows = table()
    l2h, l2l = ln2_parts()
    out = ["// Generated by gen_logtab.py: tables of the binary64 logarithm of the window",
           "// kernels (Tang's table-driven reduction, reciprocal form). Do not edit.",
           "#pragma once", "", "namespace fskmc {", "",
           f"constexpr double LOG_LN2_HI = {l2h.hex()};",
           f"constexpr double LOG_LN2_LO = {l2l.hex()};", "",
           "// {invc, -log(invc) hi, -log(invc) lo} for the 128 reduction intervals",
           "__device__ const double LOG_TAB[128][3] = {"]
    for inv, hi, lo in rows:
        out.append(f"    {{{inv.hex()}, {hi.hex()}, {lo.hex()}}},")
    out += ["};", "", "}  // namespace fskmc", ""]
    with open(os.path.join(HERE, "fskmc_logtab.h"), "w") as f:
        f.write("\n".join(out))


if __name__ == "__main__":
    main()

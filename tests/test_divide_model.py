"""An exact model of the window kernels' binary64 divide without a divide
instruction (div_int: a 64-bit reciprocal of the divisor's significand from
a binary32 seed, two integer Newton-Raphson steps, the quotient estimate
corrected by the exact remainder and rounded to nearest-even), in Python
integers with the kernels' 64-bit wrap-around, checked against the correctly
rounded quotient. The seed is also moved by +-2^-22 (more than the binary32
reciprocal's error on the 24-bit truncated significand), so the argument
that two Newton steps leave the estimate at most a unit below the true
quotient holds with margin. The GPU test compares the device divide with the
hardware divide bit for bit (test_integer_divide_matches_hardware)."""
import random
import struct
from fractions import Fraction

M64 = (1 << 64) - 1


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def frombits(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def umulhi(a, b):
    return ((a & M64) * (b & M64)) >> 64


def s64(x):
    x &= M64
    return x - (1 << 64) if x >> 63 else x


def div_model(a, b, seed_err=0.0, newton_steps=2, nearest=True):
    """(quotient, slow): slow marks operands or quotients outside the
    normal range, which the kernels hand to the hardware divide."""
    A, B = bits(a), bits(b)
    ea, eb = A >> 52, B >> 52
    FRAC = (1 << 52) - 1
    ma, mb = (A & FRAC) | (1 << 52), (B & FRAC) | (1 << 52)
    # seed: the binary32 reciprocal of the divisor's leading 24 significand bits, as rf 2^64
    mf = struct.unpack("<f", struct.pack("<I", 0x3F800000 | ((B >> 29) & 0x7FFFFF)))[0]
    rf = f32(1.0 / mf)
    if seed_err:
        rf = f32(rf * (1 + seed_err))
    rb = struct.unpack("<I", struct.pack("<f", rf))[0]
    X = M64 if (rb >> 23) >= 127 else (((rb & 0x7FFFFF) | 0x800000) << 40)
    for _ in range(newton_steps):
        hi = umulhi(mb, X)
        lo = (mb * X) & M64
        T = ((hi << 12) | (lo >> 52)) & M64  # (mb X) >> 52, mod 2^64
        E = s64(-T)                           # (2^116 - mb X) >> 52, signed
        corr = umulhi(X, -E if E < 0 else E)
        X = (X - corr - 1) & M64 if E < 0 else (X + corr) & M64
    ge = ma >= mb
    e = ea - eb + (1023 if ge else 1022)
    hi = umulhi(ma, X)
    lo = (ma * X) & M64
    Q = hi if ge else (((hi << 1) | (lo >> 63)) & M64)
    R = s64(((ma << (52 if ge else 53)) & M64) - Q * mb)
    if R < 0:
        Q -= 1
        R += mb
    for _ in range(2):
        if R >= mb:
            Q += 1
            R -= mb
    R2 = R << 1
    if nearest and (R2 > mb or (R2 == mb and (Q & 1))):  # (an exact half cannot occur in a quotient)
        Q += 1
    if Q == 1 << 53:
        Q = 1 << 52
        e += 1
    slow = ea == 0 or ea >= 2047 or eb == 0 or eb >= 2047 or e < 1 or e > 2046 or R < 0 or R >= mb
    return frombits((e << 52) | (Q & FRAC)), slow


def cases(seed=7, n=4000):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        a = rng.uniform(0, 40) * (1e-10 if rng.random() < 0.2 else 1)   # -log(u) and beyond
        b = 10 ** rng.uniform(-6, 8)                                    # total rates
        if a > 0:
            out.append((a, b))
    for _ in range(400):
        b = 10 ** rng.uniform(-3, 5)
        out += [(b, b), (frombits(bits(b) - 1), b), (frombits(bits(b) + 1), b)]  # exact, just below, just above
    for m in range(64):
        b = frombits((1023 << 52) | (m << 29))             # significands at the seed's truncation edge
        out += [(1.7, b), (1.0, b), (1.3, frombits((1023 << 52) | ((1 << 52) - 1 - m)))]
    return out


def test_divide_model_is_correctly_rounded():
    cs = cases()
    n = slow = 0
    for err in (0.0, 2.0 ** -22, -(2.0 ** -22)):
        for a, b in cs:
            q, s = div_model(a, b, err)
            if s:
                slow += 1
                continue
            n += 1
            assert q == float(Fraction(a) / Fraction(b)), (a, b, err)
    assert n > 10000 and slow < n // 50


def test_planted_mistakes_are_caught():
    """One Newton step leaves the estimate too far from the quotient: the
    exact remainder flags most cases for the hardware divide. Truncating
    instead of rounding to nearest gives wrong quotients."""
    cs = cases(seed=11, n=1000)
    slow = sum(div_model(a, b, 0.0, newton_steps=1)[1] for a, b in cs)
    assert slow > len(cs) // 2
    wrong = 0
    for a, b in cs:
        q, s_ = div_model(a, b, nearest=False)
        if not s_ and q != float(Fraction(a) / Fraction(b)):
            wrong += 1
    assert wrong > len(cs) // 4

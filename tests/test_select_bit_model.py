"""An exact model of the member search's select-bit (the position of the
r-th set bit of a 32-bit membership word, found branch-free: byte popcounts
by the SWAR bit-count steps, their running sums by one multiply, the byte by
a bytewise compare, then the nibble and a 2-bit table of positions within a
nibble), checked against the plain definition on every r of many words. The
GPU parity tests check the device function through the lattices it picks."""
import random

M32 = 0xFFFFFFFF


def nibble_table():
    """4 words of 16 2-bit entries: entry 4 n + r = position of the r-th set
    bit of the nibble n."""
    w = [0, 0, 0, 0]
    for n in range(16):
        r = 0
        for b in range(4):
            if (n >> b) & 1:
                idx = 4 * n + r
                w[idx >> 4] |= b << (2 * (idx & 15))
                r += 1
    return w


NS = nibble_table()


def popc(x):
    return bin(x & M32).count("1")


def select_model(m, r):
    c = (m - ((m >> 1) & 0x55555555)) & M32
    c = ((c & 0x33333333) + ((c >> 2) & 0x33333333)) & M32
    c = (c + (c >> 4)) & 0x0F0F0F0F
    p = (c * 0x01010101) & M32                      # byte i: set bits in bytes 0..i
    gt = (((p | 0x80808080) - (r + 1) * 0x01010101) & M32) & 0x80808080
    b = min(4 - popc(gt), 3)                        # whole bytes before the bit
    sh = 8 * b
    before = (((p << 8) & M32) >> sh) & 0xFF
    v = (m >> sh) & 0xFF
    rr = r - before
    c4 = popc(v & 15)
    hi = rr >= c4
    nib = (v >> 4) if hi else (v & 15)
    rr -= c4 if hi else 0
    idx = (nib * 4 + rr) & 63
    word = NS[idx >> 4]
    return sh + (4 if hi else 0) + ((word >> (2 * (idx & 15))) & 3)


def select_plain(m, r):
    seen = 0
    for pos in range(32):
        if (m >> pos) & 1:
            if seen == r:
                return pos
            seen += 1
    raise ValueError


def words():
    rng = random.Random(5)
    out = [M32, 1, 1 << 31, 0x80000001, 0x00FF00FF, 0xFF00FF00, 0x0F0F0F0F, 0xF0F0F0F0, 0x01010101, 0x80808080]
    out += [1 << i for i in range(32)]
    out += [rng.getrandbits(32) for _ in range(3000)]
    out += [rng.getrandbits(32) & rng.getrandbits(32) & rng.getrandbits(32) for _ in range(1000)]  # sparse
    out += [rng.getrandbits(32) | rng.getrandbits(32) | rng.getrandbits(32) for _ in range(1000)]  # dense
    return [w for w in out if w]


def test_select_bit_matches_its_definition():
    n = 0
    for m in words():
        for r in range(popc(m)):
            assert select_model(m, r) == select_plain(m, r), (hex(m), r)
            n += 1
    assert n > 50000


def test_nibble_table_entries():
    for n in range(16):
        bits = [b for b in range(4) if (n >> b) & 1]
        for r, b in enumerate(bits):
            idx = 4 * n + r
            assert (NS[idx >> 4] >> (2 * (idx & 15))) & 3 == b

"""The arithmetic behind the verification kernel's packed level tests
(Algorithm 1's tests on the first four chunks, k = 32), checked on the CPU.

The kernel keeps the cumulative disagreements D_i = 32 (i + 1) - m_i of
levels 0..3 in the 16-bit halves of two 32-bit words and decides each test
with one add per word, reading bit 15 of each half:

  prune_i  (m_i <  mm_i)   <=>  D_i > dmax_i,  dmax_i = 32 (i + 1) - mm_i
  conc_i   (m_i >= clo_i)  <=>  D_i < e_i,     e_i = 32 (i + 1) - clo_i + 1

with dmax_i clamped to [-1, 0x7fff] and e_i to [0, 0x7fff].  This file
restates that packing in Python and checks it against the tests written
the plain way, with thresholds inside, at and beyond the ends of their
ranges (including the sentinel values a table uses for "never" and
"always"), so that the clamping argument -- no carry or borrow leaves a
half -- is pinned by brute force rather than by reading."""
import random

MASK = 0x80008000
U32 = 0xFFFFFFFF


def pack(levels, lite, mm, clo):
    """Per-word constants: kp (prune adder) and ec (concentration minuend)."""
    kp, ec = [0, 0], [0, 0]
    for i in range(4):
        w, h = i >> 1, (i & 1) * 16
        dmax, e = 0x7FFF, 0
        if i < levels:
            dmax = max(-1, min(0x7FFF, 32 * (i + 1) - mm[i]))
            if not lite:
                e = max(0, min(0x7FFF, 32 * (i + 1) - clo[i] + 1))
        kp[w] |= (0x7FFF - dmax) << h
        ec[w] |= (0x7FFF + e) << h
    return kp, ec


def packed_bits(kp, ec, d):
    """prune and concentration bits of levels 0..3 from per-chunk disagreements d."""
    e1 = d[0] + d[1]
    e2 = e1 + d[2]
    w = [(d[0] | e1 << 16) & U32, (e2 | (e2 + d[3]) << 16) & U32]
    p = [((w[i] + kp[i]) & U32) & MASK for i in range(2)]
    c = [((ec[i] - w[i]) & U32) & MASK for i in range(2)]
    prune = conc = 0
    for i in range(4):
        bit = 0x8000 << ((i & 1) * 16)
        prune |= (1 if p[i >> 1] & bit else 0) << i
        conc |= (1 if c[i >> 1] & bit else 0) << i
    return prune, conc


def plain_bits(levels, lite, mm, clo, d):
    prune = conc = 0
    m = 0
    for i in range(4):
        m += 32 - d[i]
        if i < levels:
            prune |= (m < mm[i]) << i
            if not lite:
                conc |= (m >= clo[i]) << i
    return prune, conc


def threshold(i, rng):
    n = 32 * (i + 1)
    return rng.choice([-2 ** 31, -7, -1, 0, 1, 2, rng.randint(0, n), n - 1, n, n + 1, n + 2, 2 ** 31 - 1])


def test_packed_tests_equal_the_plain_tests():
    rng = random.Random(7)
    cases = 0
    for _ in range(3000):
        levels = rng.choice([1, 2, 3, 4, 5, 64])
        lite = rng.random() < 0.3
        mm = [threshold(i, rng) for i in range(4)]
        clo = [threshold(i, rng) for i in range(4)]
        kp, ec = pack(levels, lite, mm, clo)
        for _ in range(60):
            d = [rng.choice([0, 32, rng.randint(0, 32)]) for _ in range(4)]
            assert packed_bits(kp, ec, d) == plain_bits(levels, lite, mm, clo, d), (levels, lite, mm, clo, d)
            cases += 1
    assert cases == 180000


def test_every_half_stays_below_two_to_the_sixteen():
    """The sums the kernel forms never carry out of a half, nor borrow into one."""
    for dmax in range(-1, 0x8000, 97):
        for D in range(0, 129):
            assert 0 <= D + (0x7FFF - dmax) < 0x10000
    for e in range(0, 0x8000, 97):
        for D in range(0, 129):
            assert 0 <= (0x7FFF + e) - D < 0x10000

"""The arithmetic scheme of the FP64 push's 64-bit fixed point, checked on
the CPU with exact Python integers (csrc/pic_fixed64.cuh states the claims):

- a product x W / 2^62 formed from three 32x32 -> 64-bit multiply-adds stays
  within 2n + 1 units over n products, with every accumulator in int64 range
  under the stated bounds, and a sum of zero products is exactly zero;
- the compensated product has no bias over the weight's low bits;
- the double -> fixed conversion from the bit pattern rounds to nearest;
- the (high, low) 32-bit word pair with a carry from the low word's old value
  holds the exact 64-bit sum in any order of the adds;
- the running sums of the Esirkepov deposit change by at most 3/4 of the
  particle's move along the axis (the slope bound behind the J tile's scale).

These run the scheme, not the kernel; the GPU parity tests run the kernel.
"""
import random
import struct
from fractions import Fraction

import numpy as np

M64 = 1 << 64


def s64(v):
    v &= M64 - 1
    return v - M64 if v >= 1 << 63 else v


def w62(W):
    return W >> 31, W & 0x7FFFFFFF


def fix_init():
    return [0, 1 << 29, 1 << 30]


def fix_mac(acc, x, w, compensate=False):
    x1, x0 = x >> 32, x & 0xFFFFFFFF
    assert -(1 << 31) <= x1 < (1 << 31) and 0 <= w[0] < (1 << 31)
    acc[0] += x1 * w[0]
    acc[1] += x1 * w[1]
    acc[2] += x0 * w[0] + ((x0 >> 1) if compensate else 0)
    assert abs(acc[0]) < 1 << 63 and abs(acc[1]) < 1 << 63 and 0 <= acc[2] < M64


def fix_result(acc):
    return s64(2 * acc[0] + (acc[1] >> 30) + (acc[2] >> 31))


def to_fixed(v, k):
    b = struct.unpack("<q", struct.pack("<d", v))[0]
    e = (b >> 52) & 0x7FF
    m = (b & 0xFFFFFFFFFFFFF) | 0x10000000000000
    sh = e - 1075 + k
    lsh, rsh = max(sh, 0), min(max(-sh, 0), 62)
    X = ((m << lsh) + ((1 << rsh) >> 1)) >> rsh
    X = 0 if e == 0 else X
    return -X if b < 0 else X


def bspline3(t):
    s = 1.0 - t
    return np.array([s ** 3 / 6, 2 / 3 - t * t + t ** 3 / 2, 2 / 3 - s * s + s ** 3 / 2, t ** 3 / 6])


def test_gather_sums_stay_in_range_and_within_2n_plus_1_units():
    rng = random.Random(1)
    worst = 0.0
    for _ in range(4000):
        n = rng.choice([1, 2, 4])
        ws = [rng.random() for _ in range(n)]
        if n > 1:  # spline weights sum to one
            t = sum(ws)
            ws = [w / t for w in ws]
        W = [min(int(round(w * 2 ** 62)), 2 ** 62 - 1) for w in ws]
        xs = [rng.choice([rng.randint(-(2 ** 60) + 1, 2 ** 60 - 1), 2 ** 60 - 1, -(2 ** 60) + 1, -1, 1])
              for _ in range(n)]
        acc = fix_init()
        for x, Wi in zip(xs, W):
            fix_mac(acc, x, w62(Wi))
        exact = sum(Fraction(x) * Wi / 2 ** 62 for x, Wi in zip(xs, W))
        worst = max(worst, float(abs(fix_result(acc) - exact)) / (2 * n + 1))
    assert worst <= 1.0


def test_zero_products_sum_to_exactly_zero():
    for n in (1, 2, 4):
        acc = fix_init()
        for _ in range(n):
            fix_mac(acc, 0, w62(3074457345618258603))
        assert fix_result(acc) == 0
        acc = fix_init()
        fix_mac(acc, 0, w62(12345), compensate=True)
        assert fix_result(acc) == 0


def test_compensated_product_is_unbiased_and_within_2_units():
    rng = random.Random(5)
    plain, comp = [], []
    for _ in range(20000):
        x = rng.randint(-(2 ** 62), 2 ** 62)
        W = rng.randint(0, 2 ** 62 - 1)
        exact = Fraction(x) * W / 2 ** 62
        for out, c in ((plain, False), (comp, True)):
            acc = fix_init()
            fix_mac(acc, x, w62(W), compensate=c)
            out.append(float(fix_result(acc) - exact))
    assert abs(np.mean(plain) + 0.5) < 0.02  # the dropped low x low term: half a unit low
    assert abs(np.mean(comp)) < 0.02
    assert max(abs(e) for e in comp) <= 2.0


def test_to_fixed_rounds_to_nearest():
    rng = random.Random(2)
    for _ in range(20000):
        k = rng.randint(-60, 120)
        v = rng.uniform(-1, 1) * 2.0 ** (61 - k) * rng.choice([1, 1e-3, 1e-9])
        X = to_fixed(v, k)
        assert abs(X - Fraction(v) * Fraction(2) ** k) <= Fraction(1, 2)
    assert to_fixed(0.0, 62) == 0 and to_fixed(-0.0, 62) == 0 and to_fixed(5e-320, 1000) == 0


def test_word_pair_with_carry_is_exact_in_any_order():
    rng = random.Random(3)
    mask = (1 << 32) - 1
    for _ in range(300):
        xs = [rng.randint(-(2 ** 54), 2 ** 54) for _ in range(rng.randint(1, 400))]
        rng.shuffle(xs)
        hi = lo = 0
        for X in xs:
            u = X & (M64 - 1)
            l, h = u & mask, u >> 32
            old = lo
            lo = (lo + l) & mask
            hi = (hi + h + (1 if ((old + l) & mask) < old else 0)) & mask
        assert s64((hi << 32) | lo) == sum(xs)


def test_deposit_running_sums_move_at_most_three_quarters_of_the_move():
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(20000):
        x0 = rng.uniform(0, 1)
        d = rng.uniform(-1, 1) * rng.choice([1.0, 1e-3, 1e-7])
        x1 = x0 + d
        c1 = int(np.floor(x1))
        # the Esirkepov window: nodes -2..3 (array index node + 2); a particle
        # in cell c has weights on the nodes c - 1 .. c + 2
        S0 = np.zeros(6)
        S1 = np.zeros(6)
        S0[1:5] = bspline3(x0)
        S1[c1 + 1:c1 + 5] = bspline3(x1 - c1)
        run = np.cumsum(S1 - S0)
        worst = max(worst, np.abs(run).max() / abs(d))
    assert worst <= 0.75 + 1e-6

"""CPU check of the arithmetic behind the tensor-core FP64 emulation of the deflation products
(reading 21; the paper computes these products in plain arithmetic, Sec. 5.4).

An integer model of the splitting, written here independently of the CUDA code: each operand row
(left) or column (right) is scaled by a power of two to entries below 1/2 and cut into seven
balanced base-256 digits; slice products are grouped by g = s + t <= 7; groups 0..4 are summed
exactly, groups 5..7 in FP32; the exact part and the tail are folded once into FP64.  The model's
result is compared with the exact rational value of sum_i a_i b_i, against the bound stated for
the method: 2^-52 (max|a| sum|b| + sum|a| max|b|) plus one FP64 rounding of the result.  A second
check pins the read-out interval: with the worst digits (all 128, one sign) the exact groups of
one read-out stay within 2^24, so the FP32 sums in tensor memory are exact integers.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

NS = 7        # slices per operand
NG = 8        # slice groups g = s + t <= 7
NEXACT = 5    # groups 0..4 exact


def scale_exp(v):
    """e with |x| < 2^(e-1) for every entry of v (0 for an all-zero vector)."""
    m = float(np.max(np.abs(v))) if len(v) else 0.0
    if m == 0.0:
        return 0
    _, E = math.frexp(m)          # m = f 2^E, f in [1/2, 1)  =>  m < 2^E
    return E + 1


def digits(x, e):
    """Balanced base-256 digits d_0..d_6 of |x| 2^-e truncated after 56 bits, sign applied."""
    F = int(math.ldexp(abs(x), 8 * NS - e))      # exact scaling, truncation toward zero
    d = [0] * NS
    for s in range(NS - 1, 0, -1):
        dd = F & 255
        if dd >= 128:
            dd -= 256
        d[s] = dd
        F = (F - dd) >> 8
    d[0] = F
    return [-v for v in d] if x < 0 else d


def small_digits(v):
    """One exact digit per entry when every entry is an integer below 256 times a common 2^e."""
    nz = [x for x in v if x != 0.0]
    if not nz:
        return 0, [0] * len(v)
    def lsb_exp(x):       # exponent of the lowest set bit of x
        m, E = math.frexp(x)
        mant = int(math.ldexp(abs(m), 53))
        return E - 53 + (mant & -mant).bit_length() - 1
    e = min(lsb_exp(x) for x in nz)
    d = [int(math.ldexp(x, -e)) for x in v]
    if any(abs(q) >= 256 or math.ldexp(q, e) != x for q, x in zip(d, v)):
        return None
    return e, d


def emulated_dot(a, b, small_b=False):
    """sum_i a_i b_i by the splitting model: returns (FP64 result, max |exact group| in units)."""
    ea = scale_exp(a)
    da = [digits(x, ea) for x in a]
    if small_b:
        eb, db = small_digits(b)
        db = [[q] for q in db]
        unit_shift = 8     # product of slice s and the integer digit: unit 2^-8(s+1)
    else:
        eb = scale_exp(b)
        db = [digits(x, eb) for x in b]
        unit_shift = 16    # product of slices s, t: unit 2^-8(s+t+2)
    nb = len(db[0])
    exact = [0] * NEXACT               # integer group sums in units 2^-(8g + unit_shift)
    tail = np.float32(0.0)
    for i in range(len(a)):
        for s in range(NS):
            for t in range(nb):
                g = s + t
                if g >= NG:
                    continue
                p = da[i][s] * db[i][t]
                if g < NEXACT:
                    exact[g] += p
                else:
                    tail = np.float32(tail + np.float32(math.ldexp(p, -(8 * g + unit_shift))))
    T = 0
    for g in range(NEXACT):
        T = T * 256 + exact[g]
    val = math.ldexp(float(T), -(8 * (NEXACT - 1) + unit_shift)) + float(tail)   # one conversion of T
    return math.ldexp(val, ea + eb), max(abs(v) for v in exact)


def bound(a, b):
    a, b = np.abs(a), np.abs(b)
    return a.max() * b.sum() + a.sum() * b.max()


def exact_dot(a, b):
    return sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))


CASES = [("gauss", 1), ("gauss", 7), ("gauss", 200), ("gauss", 3000), ("spread", 200), ("spread", 3000),
         ("tiny-huge", 64), ("near-max", 500)]


@pytest.mark.parametrize("kind,n", CASES)
def test_emulated_dot_within_stated_bound(kind, n):
    r = np.random.default_rng(n + len(kind))
    a, b = r.standard_normal(n), r.standard_normal(n)
    if kind == "spread":
        a *= np.exp(r.uniform(-8, 8, n))
        b *= np.exp(r.uniform(-8, 8, n))
    elif kind == "tiny-huge":
        a *= 10.0 ** r.integers(-30, 30, n)
        b *= 10.0 ** r.integers(-30, 30, n)
    elif kind == "near-max":
        a = np.where(r.random(n) < 0.5, 1.0, -1.0) * (1.0 - 2.0 ** -40)
        b = np.full(n, 0.999999999)
    got, _ = emulated_dot(a, b)
    ex = exact_dot(a, b)
    err = abs(Fraction(got) - ex)
    lim = Fraction(2.0 ** -52 * bound(a, b)) + Fraction(2.0 ** -53) * abs(ex)
    assert err <= lim, "error %.3e > %.3e" % (float(err), float(lim))


def test_small_integer_right_operand_is_exact_slice():
    r = np.random.default_rng(5)
    a = r.standard_normal(400)
    b = r.choice([1.0, -1.0, 0.0], 400)          # Z(4) components
    assert small_digits(b) is not None
    got, _ = emulated_dot(a, b, small_b=True)
    ex = exact_dot(a, b)
    # only the left operand's truncation and the final rounding remain
    lim = Fraction(2.0 ** -54 * np.abs(a).max() * np.abs(b).sum()) + Fraction(2.0 ** -53) * abs(ex)
    assert abs(Fraction(got) - ex) <= lim


def test_readout_interval_keeps_exact_groups_within_fp32_integers():
    """Worst case: every digit 128 with one sign.  Seven-slice operands, read-out every 6 chunks of
    32 (at most 5 pairs in an exact group); one-slice Z(4) operand (digit magnitude below 2),
    every 2048 chunks.  All exact-group sums stay within 2^24."""
    for pairs, dB, chunks in ((5, 128, 6), (1, 2, 2048)):
        worst = chunks * 32 * pairs * 128 * dB
        assert worst <= 2 ** 24
        assert (chunks + 1) * 32 * pairs * 128 * dB > 2 ** 24      # the interval is the largest such
    # and the model agrees on an adversarial input of that length (seven slices on both sides)
    n = 6 * 32
    a = np.full(n, math.ldexp(255.0 / 256.0, -1) * (1 - 2.0 ** -30))
    _, worst_group = emulated_dot(a, a)
    assert worst_group <= 2 ** 24

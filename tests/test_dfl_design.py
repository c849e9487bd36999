"""The double-float arithmetic of FQ_DF32 (values hi + lo of two FP32 numbers), modelled on CPU
with every FP32 operation rounded once, exactly as the GPU's explicitly rounded instructions are:
the fused multiply-add a*b + c (Dekker's exact product by FMA, Knuth's two-sum, a fast
renormalisation) is accurate to 2^-45 of (|a b| + |c|) (worst seen about 2^-46.3: the pair holds
48 bits, the rounded cross terms and sums cost one or two) and leaves |lo| within half an ulp of
hi.  (The CUDA path is checked against the oracle by the GPU tests.)"""
import math
import random
from fractions import Fraction

import pytest


def rnd32(q):
    """The binary32 value nearest the rational q (ties to even), as a Python float."""
    q = Fraction(q)
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = math.floor(math.log2(q.numerator) - math.log2(q.denominator))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    scale = Fraction(2) ** (e - 23)              # 24-bit significand: q / scale in [2^23, 2^24)
    m = q / scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * float(fl * scale)


def fadd(a, b):
    return rnd32(Fraction(a) + Fraction(b))


def fsub(a, b):
    return rnd32(Fraction(a) - Fraction(b))


def fmul(a, b):
    return rnd32(Fraction(a) * Fraction(b))


def fma(a, b, c):
    return rnd32(Fraction(a) * Fraction(b) + Fraction(c))


def dfl_of(x):
    h = rnd32(x)
    return h, rnd32(Fraction(x) - Fraction(h))


def dfl_fma(a, b, c):
    """a * b + c for double-floats, step for step as the kernels compute it."""
    p = fmul(a[0], b[0])
    pe = fma(a[0], b[0], -p)                      # exact: a.h b.h = p + pe
    pe = fma(a[0], b[1], fma(a[1], b[0], pe))     # cross terms (a.l b.l is below 2^-48)
    s = fadd(p, c[0])                             # two-sum of p and c.h
    bb = fsub(s, p)
    se = fadd(fsub(p, fsub(s, bb)), fsub(c[0], bb))
    se = fadd(se, fadd(pe, c[1]))
    h = fadd(s, se)                               # fast renormalisation
    return h, fsub(se, fsub(h, s))


def value(x):
    return Fraction(x[0]) + Fraction(x[1])


def test_rnd32_matches_numpy_float32():
    """The single rounding equals numpy's float64 -> float32 cast wherever the float64 input is
    the exact value (so no double rounding can occur)."""
    np = pytest.importorskip("numpy")
    rng = random.Random(1)
    for _ in range(3000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        assert rnd32(x) == float(np.float32(x))


def test_two_product_and_two_sum_are_exact():
    rng = random.Random(2)
    for _ in range(2000):
        a, b = rnd32(rng.uniform(-4, 4)), rnd32(rng.uniform(-4, 4))
        p = fmul(a, b)
        assert Fraction(p) + Fraction(fma(a, b, -p)) == Fraction(a) * Fraction(b)
        s = fadd(a, b)
        bb = fsub(s, a)
        err = fadd(fsub(a, fsub(s, bb)), fsub(b, bb))
        assert Fraction(s) + Fraction(err) == Fraction(a) + Fraction(b)


@pytest.mark.parametrize("spread", [0, 10, 30])
def test_dfl_fma_precision_and_normalisation(spread):
    """|(a b + c) - dfl_fma(a, b, c)| <= 2^-45 (|a b| + |c|), including heavy cancellation
    between a b and c, and the result is normalised: |lo| <= ulp(hi) / 2."""
    rng = random.Random(3 + spread)
    worst = 0.0
    for _ in range(1500):
        a = dfl_of(rng.uniform(-2, 2) * 2.0 ** rng.randint(-spread, spread))
        b = dfl_of(rng.uniform(-2, 2) * 2.0 ** rng.randint(-spread, spread))
        if rng.random() < 0.3:   # c close to -a b: the exact result is far below |a b|
            c = dfl_of(-float(value(a) * value(b)) * (1 + rng.uniform(-1e-6, 1e-6)))
        else:
            c = dfl_of(rng.uniform(-2, 2) * 2.0 ** rng.randint(-spread, spread))
        exact = value(a) * value(b) + value(c)
        r = dfl_fma(a, b, c)
        scale = abs(value(a) * value(b)) + abs(value(c))
        err = abs(value(r) - exact) / scale
        worst = max(worst, float(err))
        assert err <= Fraction(2) ** -45
        if r[0] != 0:
            ulp = 2.0 ** (math.floor(math.log2(abs(r[0]))) - 23)
            assert abs(r[1]) <= ulp / 2
    assert worst > 0  # the test can tell an exact result from a rounded one

"""The arithmetic the FP64 emulation (FQ_OZAKI) rests on, checked on CPU by brute force:
fixed-point digits taken from the FP64 bit pattern by rounding shifts, their bounds and
reconstruction error, and the exactness of the FP32 group sums over one drain interval.
(The CUDA kernels themselves are checked against the oracle by the GPU tests.)"""
import struct

import numpy as np


def bits_digits(x, E, nslices=6):
    """R = x 2^(48-E) rounded (half away from zero) from the significand and exponent of x, then
    digits by rounding shifts of 8 bits - the integer procedure of the slicing kernels."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    be = (b >> 52) & 0x7FF
    sh = 1027 + E - be
    R = 0
    if be != 0 and sh < 64:
        m = (b & ((1 << 52) - 1)) | (1 << 52)
        R = (m + (1 << (sh - 1))) >> sh
        if b >> 63:
            R = -R
    ds = []
    for q in range(nslices):
        s = 40 - 8 * q
        if s > 0:
            d = (R + (1 << (s - 1))) >> s
            R -= d << s
        else:
            d = R
        ds.append(d)
    return ds


def row_exponent(mx):
    if mx == 0:
        return 0
    b = struct.unpack("<Q", struct.pack("<d", mx))[0]
    return max(((b >> 52) & 0x7FF) - 1023 + 2, -960)


def test_digits_bounds_and_reconstruction():
    rng = np.random.default_rng(7)
    for trial in range(400):
        row = rng.normal(size=32) * 10.0 ** rng.uniform(-40, 40)
        row[trial % 32] = 0.0
        E = row_exponent(float(np.max(np.abs(row))))
        for x in row:
            ds = bits_digits(float(x), E)
            assert max(abs(d) for d in ds) <= 128
            rec = sum(d * 2.0 ** (-8 * (q + 1)) for q, d in enumerate(ds)) * 2.0 ** E
            assert abs(rec - x) <= 2.0 ** (E - 49) * (1 + 1e-12)
            # every slice is an integer times 2^-8(q+1) with at most 8 significant bits: exact in BF16
            for q, d in enumerate(ds):
                v = np.float32(d * 2.0 ** (-8 * (q + 1)))
                assert float(v) == d * 2.0 ** (-8 * (q + 1)) and abs(d) <= 256


def test_group_sums_are_exact_over_a_drain_interval():
    """Worst case: every digit at its bound and every product of one sign.  Complex products
    take 256 products per pair per 128 values of k, real ones 256 per 256 values; the groups
    a + b = 0, 1, 2 hold 1, 2 and 3 pairs.  FP32 sums of such integers stay exact below 2^24."""
    for pairs in (1, 2, 3):
        worst = pairs * 128 * 128 * 256
        assert worst < 2 ** 24
        terms = np.full(pairs * 256, 128 * 128, dtype=np.float32)
        acc = np.float32(0)
        for t in terms:
            acc = np.float32(acc + t)
        assert int(acc) == worst
    # random digits: the FP32 running sum equals the integer sum
    rng = np.random.default_rng(3)
    for _ in range(50):
        d1 = rng.integers(-128, 129, size=3 * 256)
        d2 = rng.integers(-128, 129, size=3 * 256)
        acc = np.float32(0)
        for p in (d1 * d2).astype(np.float32):
            acc = np.float32(acc + p)
        assert int(acc) == int(np.sum(d1.astype(np.int64) * d2.astype(np.int64)))

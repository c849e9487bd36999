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


def _digits_matrix(X, E, nslices=6):
    """Digits of every entry of X (rows share exponent E[i]) as int64 arrays [q][i][k]."""
    m, k = X.shape
    out = np.zeros((nslices, m, k), dtype=np.int64)
    for i in range(m):
        for j in range(k):
            out[:, i, j] = bits_digits(float(X[i, j]), int(E[i]), nslices)
    return out


def _emulated_product(A, B, max_pair_sum=5):
    """A B from 6 digit slices per operand: A's rows and B's columns each carry their own power
    of two, the slice pairs (q, r) with q + r <= max_pair_sum (21 pairs for 5) are summed exactly
    over k in integers, then scaled.  This is the product the emulation's integer part computes."""
    EA = np.array([row_exponent(float(np.max(np.abs(r)))) for r in A])
    EB = np.array([row_exponent(float(np.max(np.abs(c)))) for c in B.T])
    dA = _digits_matrix(A, EA)
    dB = _digits_matrix(B.T, EB)
    C = np.zeros((A.shape[0], B.shape[1]))
    npairs = 0
    for s in range(max_pair_sum, -1, -1):  # small terms first
        for q in range(s + 1):
            r = s - q
            C += (dA[q] @ dB[r].T).astype(np.float64) * 2.0 ** (-8 * (q + 1) - 8 * (r + 1))
            npairs += 1
    assert npairs == (max_pair_sum + 1) * (max_pair_sum + 2) // 2
    return C * np.exp2(EA[:, None] + EB[None, :]), EA, EB


def _normwise_bound(k, EA, EB):
    """Per entry: k terms, each off by at most 2^-49 (reconstruction of either factor, scaled
    by the other's |.| < 1/2) plus the dropped pairs q + r >= 6 (5 pairs of 2^-50 and smaller),
    in units of 2^(EA_i + EB_j): k * 7 * 2^-50 * (1 + 2^-7), and the FP64 rounding of the final
    scaled sums."""
    return k * 7.0 * 2.0 ** -50 * (1 + 2.0 ** -7) * np.exp2(EA[:, None] + EB[None, :]) * (1 + 1e-12)


def test_pair_truncation_matches_exact_product():
    """On a small case, against the exact rational product: the 21-pair emulation stays inside
    its normwise bound, and dropping the a + b = 5 pairs (15 pairs) is visibly worse."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    m, k, n = 6, 64, 5
    A = rng.normal(size=(m, k)) * np.exp2(rng.integers(-20, 20, size=(m, 1)))
    B = rng.normal(size=(k, n)) * np.exp2(rng.integers(-20, 20, size=(1, n)))
    C, EA, EB = _emulated_product(A, B)
    exact = np.array([[float(sum(Fraction(float(A[i, t])) * Fraction(float(B[t, j])) for t in range(k)))
                       for j in range(n)] for i in range(m)])
    err = np.abs(C - exact)
    bound = _normwise_bound(k, EA, EB)
    assert np.all(err <= bound)
    # without the a + b = 5 pairs the error grows by about 2^8
    C15, _, _ = _emulated_product(A, B, max_pair_sum=4)
    unit = np.exp2(EA[:, None] + EB[None, :])
    assert np.max(np.abs(C15 - exact) / unit) > 64 * np.max(err / unit)


def test_pair_truncation_on_propagator_shaped_operands():
    """A rescaled GOE operator (spectrum in [-1, 1]) times a unitary block, k = 128: the emulated
    product agrees with a long-double product inside the same bound.  Six 8-bit slices keep 48
    bits relative to each row's scale, so one product is some tens of times less accurate than a
    plain FP64 product (below 1e-13 here, against about 1e-16), far inside the 1e-10 the
    FP64-level paths are held to for a whole U_T."""
    rng = np.random.default_rng(12)
    k = 128
    g = rng.normal(size=(k, k))
    H = (g + g.T) / np.sqrt(2 * k) / 2.0
    Q, _ = np.linalg.qr(rng.normal(size=(k, 16)))
    C, EA, EB = _emulated_product(H[:16], Q)
    ref = (H[:16].astype(np.longdouble) @ Q.astype(np.longdouble)).astype(np.float64)
    ref_err = k * np.finfo(np.longdouble).eps * (np.abs(H[:16]) @ np.abs(Q))
    assert np.all(np.abs(C - ref) <= _normwise_bound(k, EA, EB) + ref_err)
    assert np.max(np.abs(C - ref)) < 1e-13

"""The band form of the tridiagonal step (FQ_OZAKI on a tridiagonal plan, csrc/band.cu), checked in
FP64 on CPU against the oracle, free of the emulation's rounding:

  * P_m = e^{-i beta h} sum_k c_k T_k(Omega~_m) (Eqs. 10 and 12) is a band matrix with 2L + 1
    diagonals, and row i of it is what the kernel forms: Clenshaw's recurrence on the basis vector
    e_i in the real gauge frame, on a 96-row window centred on i (zero beyond it), rotated back by
    e^{i theta_i} ... e^{-i theta_k};
  * chaining X_m = P_m X_{m-1} reproduces the oracle's step-by-step recurrence;
  * the tile window of 64 operator rows [i0, i0 + 64), state columns [i0 - kh, i0 + 64 + kh)
    (kh = L rounded up to a multiple of 8), holds every row's band, and each row's window
    positions land inside it;
  * one drain per tile keeps the three exact FP32 sums exact (3 pairs x 2^14 x 320 < 2^24);
  * the FP32 cut of a double-float state entry into its 8-bit digits (k_band_slice) is exact to
    2^-49 of the row scale, with digits that keep the tensor-core sums exact."""
import math
from fractions import Fraction

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o
from test_gauge_design import clenshaw, gauge

WIN, CENTRE, BN = 96, 48, 64


def window(L):
    """The product's K half-width and tile width for a series of L products: kh = L rounded up
    to a multiple of 8 (at most 48), so the window is a whole number of 16-row K stages."""
    kh = min(48, -(-L // 8) * 8)
    return kh, BN + 2 * kh


def band_rows(d, e_real, theta, coeffs, phase, n):
    """The kernel's formation of P_m, row by row: v = P(Omega') e_i on the window [i - 48, i + 48)
    (operator zero outside [0, n) and outside the window), then P[i][k] = phase e^{i theta_i} v_k
    e^{-i theta_k}."""
    P = np.zeros((n, n), complex)
    for i in range(n):
        w0 = i - CENTRE
        ks = np.arange(w0, w0 + WIN)
        inside = (ks >= 0) & (ks < n)
        dw = np.where(inside, d[np.clip(ks, 0, n - 1)], 0.0)
        ew = np.zeros(WIN)               # 2 Omega'[k+1][k] -> coupling of positions p and p + 1
        ok = inside[:-1] & inside[1:]
        ew[:-1][ok] = e_real[np.clip(ks[:-1], 0, n - 2)][ok]
        v = np.zeros((WIN, 1), complex)
        v[CENTRE] = 1.0
        s = clenshaw(dw, ew[:-1], v, coeffs)[:, 0]
        k = ks[inside]
        P[i, k] = phase * np.exp(1j * theta[i]) * s[inside] * np.exp(-1j * theta[k])
    return P


def dimer_step(nb=150, M=40, m=7, drv=None):
    h0d, h0o, h1d = fi.dimer_matrices(nb, 1.0, U=2.0 / nb)
    drv = drv or fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = o.plan_for_drive_tridiag(h0d, h0o, h1d, drv, M)
    k_low = o.commutator_tridiag(h0o, h1d)
    return h0d, h0o, h1d, plan, k_low, drv


def test_band_rows_are_the_step_polynomial():
    """The windowed Clenshaw rows equal the oracle's step applied to the identity, and the
    oracle's step has exactly 2L + 1 non-zero diagonals (T_k of a tridiagonal matrix)."""
    h0d, h0o, h1d, plan, k_low, _ = dimer_step()
    n = h0d.shape[0]
    m = 7
    d, lower = o.omega_tilde_tridiag(h0d, h0o, h1d, k_low, plan, m)
    assert np.max(np.abs(lower.imag)) > 0 and plan.L <= 47
    ref = o.chebyshev_step(lambda v: o.apply_tridiag(d, lower, v), np.eye(n, dtype=complex), plan.coeffs,
                           plan.phase)
    i, k = np.indices((n, n))
    assert np.all(ref[np.abs(i - k) > plan.L] == 0)
    assert np.min(np.abs(ref[np.abs(i - k) == plan.L])) > 0
    theta, e_real = gauge(lower)
    P = band_rows(d, e_real.real, theta, plan.coeffs, plan.phase, n)
    assert np.max(np.abs(P - ref)) <= 1e-14


def test_band_chain_matches_oracle():
    """X_m = P_m X_{m-1} over several steps (non-even drive) against the oracle's recurrence."""
    nb, M = 60, 16
    h0d, h0o, h1d, plan, k_low, drv = dimer_step(nb=nb, M=M)
    n = nb + 1
    x0 = fi.ginibre(n, 31)[:, :4]
    x0 /= np.linalg.norm(x0, axis=0)
    ref = o.propagate_tridiag(h0d, h0o, h1d, plan, x0, 0, 6)
    x = np.array(x0)
    for m in range(6):
        d, lower = o.omega_tilde_tridiag(h0d, h0o, h1d, k_low, plan, m)
        theta, e_real = gauge(lower)
        x = band_rows(d, e_real.real, theta, plan.coeffs, plan.phase, n) @ x
    assert np.max(np.abs(x - ref)) <= 1e-13


@pytest.mark.parametrize("n,L", [(1, 1), (41, 20), (64, 47), (700, 8), (700, 9), (700, 32), (700, 33),
                                 (10001, 39), (10001, 40), (10001, 41), (10001, 47)])
def test_tile_windows_hold_every_band(n, L):
    """Rows [i0, i0 + 64) of a tile read state columns [i0 - kh, i0 + 64 + kh) (kh = L rounded up
    to a multiple of 8); every non-zero P[i][k] (|i - k| <= L, both in [0, n)) sits in that window
    and in the row's 96-row formation window, at tile column c = k - (i0 - kh); the window's width
    is a multiple of the 16-row K stage (its start is the outer coordinate of the MN-major TMA
    boxes, free of alignment rules); the row's band columns (window positions [48 - kh, 48 + kh])
    and its zero columns (at most 64: two per lane) cover the tile row exactly once."""
    kh, kw = window(L)
    assert kw % 16 == 0 and L <= kh
    p0, p1 = max(0, CENTRE - kh), min(WIN, CENTRE + kh + 1)
    assert kw - (p1 - p0) <= 64
    tiles = -(-n // BN)
    for b in range(tiles):
        i0 = BN * b
        for i in range(i0, min(i0 + BN, n)):
            r = i - i0
            ks = np.arange(max(0, i - L), min(n, i + L + 1))
            c = ks - (i0 - kh)
            assert np.all((c >= 0) & (c < kw))
            p = ks - (i - CENTRE)
            assert np.all((p >= p0) & (p < p1)) and np.array_equal(c, r + p - CENTRE + kh)
            bw = p1 - p0
            zeros = [z if z < r else z + bw for z in range(kw - bw)]
            band = list(range(r + p0 - CENTRE + kh, r + p1 - CENTRE + kh))
            assert band[0] == r and sorted(zeros + band) == list(range(kw))


def test_one_drain_per_tile_is_exact():
    """Digits |d| <= 2^7, so a slice product is at most 2^14 units of its grid; the exact
    accumulators take at most 3 pairs, and a 160-column window gives 2 x 160 products per entry
    (real and imaginary parts of the state), so their sums stay below 2^24 units and FP32
    represents every partial sum exactly."""
    assert 3 * 2 ** 14 * (2 * window(47)[1]) < 2 ** 24
    assert 3 * 2 ** 14 * (2 * (window(47)[1] + 32)) > 2 ** 24   # two more K stages would need a second drain


def _f(x):
    return np.float32(x)


def _two_sum(a, b):
    s = _f(a + b)
    bb = _f(s - a)
    return s, _f(_f(a - _f(s - bb)) + _f(b - bb))


def _df_digits(a, b):
    """The band kernel's FP32 digit cut of a double-float value a + b (|a + b| < 1/2 in units of
    the row scale), one FP32 rounding per operation: t_q = a rounded to 2^(-8(q+1)) by adding
    and subtracting 1.5 2^(15 - 8q), a -= t_q, then a two-sum."""
    a, b = _two_sum(_f(a), _f(b))
    ts = []
    for q in range(6):
        c = _f(1.5 * 2.0 ** (15 - 8 * q))
        t = _f(_f(a + c) - c)
        ts.append(t)
        a = _f(a - t)
        a, b = _two_sum(a, b)
    return ts


def test_fp32_digit_cut_reconstructs_the_pair():
    """Each t_q is an integer of at most 128 in magnitude times 2^(-8(q+1)) (exact in BF16, and
    small enough for the exact FP32 sums), and sum t_q equals the pair's exact value to within
    2^-49, for pairs of every magnitude below 1/2."""
    rng = np.random.default_rng(17)
    for _ in range(3000):
        x = float(rng.uniform(-0.5, 0.5) * 2.0 ** -rng.integers(0, 40))
        a = np.float32(x)
        b = np.float32(x - float(a))
        ts = _df_digits(a, b)
        exact = Fraction(float(a)) + Fraction(float(b))
        for q, t in enumerate(ts):
            d = Fraction(float(t)) * Fraction(2) ** (8 * (q + 1))
            assert d.denominator == 1 and abs(d) <= 128
            assert float(np.float32(t)) == float(t)
        assert abs(sum(Fraction(float(t)) for t in ts) - exact) <= Fraction(1, 2 ** 49)

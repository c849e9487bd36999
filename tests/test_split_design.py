"""The arithmetic the split-precision paths (FQ_BF16X3, FQ_BF16X6; reading R10) rest on, checked
on CPU: BF16 rounding to nearest even, the slice recurrence x_s = bf16(x - x_0 - ... - x_{s-1}),
and the error of the sliced product with the pairs a + b < NS summed in FP32, against a bound
derived from those two facts; then the whole BF16X3 step chain on one instance of the batched
scan.  (The CUDA kernels are checked against the oracle by the GPU tests.)"""
import numpy as np
import pytest

U8 = 2.0 ** -8   # unit roundoff of BF16 (8-bit significand)
U24 = 2.0 ** -24  # unit roundoff of FP32


def bf16_rne(x):
    """float32 -> nearest BF16 value (ties to even), from the IEEE-754 bit layout: keep the top
    16 bits after adding 0x7FFF plus the lowest kept bit.  Returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def slices(x, ns):
    """x (float32) as ns BF16 slices: each is the BF16 of what the previous ones left over; the
    remainder is formed in FP32, where it is exact."""
    out, r = [], np.asarray(x, dtype=np.float32)
    for _ in range(ns):
        s = bf16_rne(r)
        out.append(s)
        r = (r - s).astype(np.float32)
    return out


def sliced_product(A, B, ns, keep=None):
    """A B from ns slices per operand, the pairs (a, b) with a + b < ns (or `keep`), each slice
    product exact in FP32 (8 x 8 significant bits), summed over k in FP32."""
    sa, sb = slices(A, ns), slices(B, ns)
    pairs = keep if keep is not None else [(a, b) for a in range(ns) for b in range(ns) if a + b < ns]
    C = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
    for a, b in sorted(pairs, key=lambda p: -(p[0] + p[1])):  # smallest terms first
        C = (C + (sa[a] @ sb[b]).astype(np.float32)).astype(np.float32)
    return C, len(pairs)


def test_bf16_rounding_matches_torch():
    """The bit-level rounding equals torch's float32 -> bfloat16 conversion (round to nearest
    even), ties and signs included."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.normal(size=100_000) * 10.0 ** rng.uniform(-20, 20, 100_000)).astype(np.float32)
    ties = (np.arange(1, 2000, dtype=np.uint32) << 16 | 0x8000).view(np.float32)  # exact halfway cases
    for v in (x, ties, -ties):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
        assert np.array_equal(bf16_rne(v), ref)


def test_slices_reconstruct():
    """|x - x_0 - ... - x_{s-1}| <= 2^(-8 s) |x| and |x_s| <= (1 + 2^-8) 2^(-8 s) |x|."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=50_000).astype(np.float32)
    for ns in (1, 2, 3):
        sl = slices(x, ns)
        rem = x.astype(np.float64) - sum(s.astype(np.float64) for s in sl)
        assert np.all(np.abs(rem) <= U8 ** ns * np.abs(x) * (1 + 1e-6))
        for q, s in enumerate(sl):
            assert np.all(np.abs(s) <= (1 + U8) * U8 ** q * np.abs(x) * (1 + 1e-6))


def _bound(ns, k, AB):
    """Per entry, in units of (|A| |B|)_ij: the product ab minus the kept pairs is the dropped
    pairs plus the two reconstruction remainders.  ns = 2: |a1 b1| + |e_a||b| + |a0 + a1||e_b|
    <= (1 + 2^-8)^2 2^-16 + 2^-16 + (1 + 2^-16) 2^-16; ns = 3: the pairs a + b >= 3 (a1 b2, a2 b1,
    a2 b2) and remainders of 2^-24.  Then the FP32 sum of k terms: k 2^-24."""
    if ns == 2:
        c = (1 + U8) ** 2 * U8 ** 2 + U8 ** 2 + (1 + U8 ** 2) * U8 ** 2
    else:
        c = 2 * (1 + U8) ** 2 * U8 ** 3 + (1 + U8) ** 2 * U8 ** 4 + U8 ** 3 + (1 + U8 ** 3) * U8 ** 3
    return (c + k * U24) * (1 + 1e-3) * AB


@pytest.mark.parametrize("ns,products", [(2, 3), (3, 6)])
def test_sliced_product_error(ns, products):
    """A rescaled operator (spectrum in [-1, 1]) times a block of unit states, k = 256: the
    sliced product stays inside its bound (X3: about 16 bits, X6: FP32 level), and the full
    product of the slices it drops is what separates it from the next slice count."""
    rng = np.random.default_rng(3)
    k = 256
    g = rng.normal(size=(k, k))
    Om = ((g + g.T) / np.sqrt(8 * k)).astype(np.float32)
    X = np.linalg.qr(rng.normal(size=(k, 64)))[0].astype(np.float32)
    exact = Om.astype(np.float64) @ X.astype(np.float64)
    AB = np.abs(Om).astype(np.float64) @ np.abs(X).astype(np.float64)
    C, npairs = sliced_product(Om, X, ns)
    assert npairs == products
    err = np.abs(C.astype(np.float64) - exact)
    assert np.all(err <= _bound(ns, k, AB))
    rel = np.max(err / AB)
    if ns == 2:
        assert 2.0 ** -22 < rel < 4 * U8 ** 2  # well below BF16's 2^-8, near 2^-16
        one, _ = sliced_product(Om, X, 1)     # hi x hi alone: BF16 level
        assert np.max(np.abs(one - exact) / AB) > 2.0 ** -12
    else:
        assert rel < 2.0 ** -18                 # FP32 level (k 2^-24 = 2^-16 is the worst case)
        three_only, _ = sliced_product(Om, X, 3, keep=[(0, 0), (0, 1), (1, 0)])
        assert np.max(np.abs(three_only - exact) / AB) > 8 * rel


def _x3_real_product(P, X):
    """P X for a real operator given as two BF16 slices (from FP64) and FP32 states X, sliced
    in turn; the three pairs a + b < 2 summed in FP32."""
    x0, x1 = slices(X, 2)
    out = (P[1] @ x0).astype(np.float32)
    out = (out + (P[0] @ x1).astype(np.float32)).astype(np.float32)
    return (out + (P[0] @ x0).astype(np.float32)).astype(np.float32)


def test_x3_chain_on_a_scan_instance():
    """The whole BF16X3 step chain modelled on CPU for the batched scan's smallest instance
    (N = 257, M = 256): operator entries in FP32 cut into slices, state slices from FP32 masters, the Chebyshev
    recurrence, Bessel sum and phase in FP32 (Eqs. 10 and 12), against the FP64 oracle on three
    basis states.  The model stays far inside the 1e-5 target of the split paths (7e-7 seen)."""
    import floquet_inputs as fi
    import oracle as o
    insts = fi.batch_scan()
    s = min(insts, key=lambda t: t.n)
    h0, h1 = fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1)
    drv = fi.Drive(0.0, s.amplitude, s.omega)
    M = 256
    plan = o.plan_for_drive_dense(h0, h1, drv, M)
    k = o.commutator_dense(h0, h1)
    cols = [0, s.n // 2, s.n - 1]
    x0 = np.zeros((s.n, len(cols)), complex)
    x0[cols, np.arange(len(cols))] = 1.0
    ref = o.propagate_dense(h0, h1, plan, x0)

    def op_slices(P):  # entries formed in FP32, then cut into two BF16 slices in FP32
        p32 = P.astype(np.float32)
        hi = bf16_rne(p32)
        return hi, bf16_rne((p32 - hi.astype(np.float32)).astype(np.float32))

    f32 = np.float32
    xr, xi = x0.real.astype(f32), x0.imag.astype(f32)
    a = plan.coeffs.astype(f32)
    for m in range(M):
        om = o.omega_tilde_dense(h0, h1, k, plan, m)
        S, A = op_slices(om.real), op_slices(om.imag)

        def apply(pr, pi):  # (S + i A)(pr + i pi)
            return ((_x3_real_product(S, pr) - _x3_real_product(A, pi)).astype(f32),
                    (_x3_real_product(S, pi) + _x3_real_product(A, pr)).astype(f32))

        p0r, p0i = xr, xi
        yr, yi = apply(p0r, p0i)
        p1r, p1i = yi, (-yr).astype(f32)                  # psi_1 = -i Y
        accr = (a[0] * p0r + a[1] * p1r).astype(f32)
        acci = (a[0] * p0i + a[1] * p1i).astype(f32)
        for l in range(1, plan.L):
            yr, yi = apply(p1r, p1i)
            nr, ni = (2 * yi + p0r).astype(f32), (-2 * yr + p0i).astype(f32)   # -2i Y + psi_{l-1}
            accr, acci = (accr + a[l + 1] * nr).astype(f32), (acci + a[l + 1] * ni).astype(f32)
            p0r, p0i, p1r, p1i = p1r, p1i, nr, ni
        ph = plan.phase
        xr = (ph.real * accr - ph.imag * acci).astype(f32)
        xi = (ph.real * acci + ph.imag * accr).astype(f32)
    err = np.max(np.abs(xr.astype(np.float64) + 1j * xi.astype(np.float64) - ref))
    assert err <= 1e-5 / 4, err

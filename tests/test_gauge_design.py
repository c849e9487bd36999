"""The algebra of the tridiagonal kernels (resident and tiled), checked in FP64 on CPU against the
oracle: the real gauge frame Omega~ = D Omega' D^+ with Omega' real symmetric, the Clenshaw
backward form of the Bessel-weighted Chebyshev sum (Eqs. 10 and 12), and the chaining of steps
through the frame changes D_m^+ D_{m-1}.  (The FP32 kernels are checked against the oracle by the
GPU tests; this pins the reformulation itself, free of FP32 rounding.)"""
import math

import numpy as np

import floquet_inputs as fi
import oracle as o


def reduced_arg(z):
    """arg(z) reduced to (-pi/2, pi/2]: the phase that makes z e^{-i phi} real (= +-|z|)."""
    out = np.where(z.real == 0, np.where(z.imag == 0, 0.0, 0.5 * math.pi), 0.0)
    nz = z.real != 0
    out[nz] = np.arctan(z.imag[nz] / z.real[nz])
    return out


def gauge(lower):
    """theta_k = sum_{j<k} phi_j and the real off-diagonal e'_k = e_k e^{-i phi_k}."""
    phi = reduced_arg(lower)
    theta = np.concatenate([[0.0], np.cumsum(phi)])
    return theta, lower * np.exp(-1j * phi)


def clenshaw(d, e_real, v, a):
    """sum_k c_k T_k(Omega') v with c_k = (-i)^k a_k, Omega' = (d, e') real symmetric tridiagonal:
    b_k = c_k v + 2 Omega' b_{k+1} - b_{k+2} (k = L..1), sum = c_0 v + Omega' b_1 - b_2."""
    def op(x):
        y = d[:, None] * x
        y[1:] += e_real[:, None] * x[:-1]
        y[:-1] += e_real[:, None] * x[1:]
        return y
    L = len(a) - 1
    c = [(-1j) ** k * a[k] for k in range(L + 1)]
    b1 = np.zeros_like(v)
    b2 = np.zeros_like(v)
    for k in range(L, 0, -1):
        b1, b2 = c[k] * v + 2 * op(b1) - b2, b1
    return c[0] * v + op(b1) - b2


def test_gauge_frame_is_real_and_similar():
    """Omega' = D^+ Omega~ D is real symmetric, its off-diagonal is +-|e_k|, and the phases lie
    in (-pi/2, pi/2] (a complex off-diagonal from the commutator term i c [H0, H1])."""
    rng = np.random.default_rng(1)
    n = 12
    d = rng.normal(size=n)
    lower = rng.normal(size=n - 1) + 1j * rng.normal(size=n - 1)
    lower[3] = 2j       # purely imaginary: phase pi/2
    lower[5] = -0.7     # negative real: phase 0, e' = -0.7
    theta, e_real = gauge(lower)
    phi = np.diff(theta)
    assert np.all((phi > -math.pi / 2) & (phi <= math.pi / 2))
    assert np.max(np.abs(e_real.imag)) <= 1e-15 and np.allclose(np.abs(e_real), np.abs(lower), atol=0, rtol=1e-15)
    om = np.diag(d).astype(complex) + np.diag(lower, -1) + np.diag(lower.conj(), 1)
    D = np.diag(np.exp(1j * theta))
    om_r = D.conj().T @ om @ D
    assert np.max(np.abs(om_r.imag)) <= 1e-15
    assert np.max(np.abs(om_r.real - (np.diag(d) + np.diag(e_real.real, -1) + np.diag(e_real.real, 1)))) <= 1e-15


def test_gauge_clenshaw_chain_matches_oracle():
    """Steps of a driven dimer with phi0 != 0 (so c_m != 0 and the off-diagonal is complex) run
    in the frame of each step by Clenshaw's recurrence equal the oracle's forward recurrence."""
    nb, M = 40, 12
    h0d, h0o, h1d = fi.dimer_matrices(nb, 1.0, U=0.05)
    drv = fi.Drive(0.3, 1.5, 3.0, 0.9)
    plan = o.plan_for_drive_tridiag(h0d, h0o, h1d, drv, M)
    k_low = o.commutator_tridiag(h0o, h1d)
    x0 = fi.ginibre(nb + 1, 7)[:, :5]
    ref = o.propagate_tridiag(h0d, h0o, h1d, plan, x0)
    v = np.array(x0)                 # frame of "step -1": the input frame (theta = 0)
    theta_prev = np.zeros(nb + 1)
    for m in range(M):
        d, lower = o.omega_tilde_tridiag(h0d, h0o, h1d, k_low, plan, m)
        assert np.max(np.abs(lower.imag)) > 0
        theta, e_real = gauge(lower)
        v = np.exp(1j * (theta_prev - theta))[:, None] * v   # D_m^+ D_{m-1}
        v = plan.phase * clenshaw(d, e_real.real, v, plan.coeffs)
        theta_prev = theta
    x = np.exp(1j * theta_prev)[:, None] * v                   # back to the original frame
    assert np.max(np.abs(x - ref)) <= 1e-13  # 4.5e-15 seen at L = 32
    # the frame change is not optional: skipping it (or its sign) is an O(1) error
    v_bad = np.array(x0)
    for m in range(M):
        d, lower = o.omega_tilde_tridiag(h0d, h0o, h1d, k_low, plan, m)
        theta, e_real = gauge(lower)
        v_bad = plan.phase * clenshaw(d, e_real.real, v_bad, plan.coeffs)
    assert np.max(np.abs(np.exp(1j * theta)[:, None] * v_bad - ref)) > 1e-3

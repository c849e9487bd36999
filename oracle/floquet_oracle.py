"""Plain FP64 CPU oracle of the Magnus-Chebyshev Floquet propagator (arXiv:1508.07621).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path; it is not part of
the product.  Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg / ``--impl reference`` arm of ``bench.py`` may import or run it.  It shares no code
with the CUDA path (it imports nothing from the package) and takes its inputs from
``floquet_inputs`` only.

Every function follows one passage of the paper and is written for checking by eye:
no blocking, fusion or reordering beyond what the cited equation states.  Library
primitives used as single steps: numpy matmul / eigvalsh / eigvals, scipy Bessel J_l and
tridiagonal eigvalsh.

Conventions (hbar = 1): h = T/M, step m = 1..M covers [(m-1)h, mh] with midpoint
tau_m = (m - 1/2)h; states are columns; U_T = U_M ... U_1 (Eq. 9 read for column
vectors: the earliest step acts first).

Readings where the paper is silent or garbled (each is also listed in the design notes):
  R1  4th-order midpoint Magnus = Eq. 14 truncated after its leading commutator, applied
      to A = -iH:  Omega_m = h H0 + (h f + h^3 f''/24) H1 + (h^3 f'/12) i[H0, H1].
  R2  E_min, E_max, beta, Delta E are spectral quantities of Omega/h, so
      Omega~ = (Omega/h - beta)/Delta E and R = h Delta E (Eqs. 11, 12).
  R4  bounds: Omega_m/h = H0 + g_m H1 + kappa_m i[H0,H1] with g_m = b_m/h, kappa_m = c_m/h.
      lambda_max(H0 + g H1) is convex in g, so its maximum over the steps is reached at the
      extreme g; the commutator part is added by Weyl's inequality (|kappa| ||[H0,H1]||_2);
      a relative margin of 1e-12 is added.  (The paper samples five instants; for cos
      drives those include the extreme f, so the leading bounds coincide up to h^2 f''.)
  R5  L = smallest integer l > R (l >= 1) with |J_{l+1}(R)| < tol.
  R7  quasienergies eps = theta/T with theta = -arg(lambda) in [-pi, pi).
  R11 piecewise-constant drives: the H1 coefficient range is widened by 10% of its span
      (or of max |f|) and frozen, so the bounds do not follow f.
  R12 6th order (Eq. 14 in full): alphas as 3-point Gauss-Legendre moments (see magnus6_omega);
      the literal midpoint-derivative alphas of Eq. 15 give only 4th order.
  R13 period averages (Eq. 17): composite Simpson over the M + 1 step boundaries (trapezoid
      for odd M).
  R14 overlap phase error (Eq. 20): the eigenvector phases and the quasienergy phase are left
      open, so Sigma_mu = |1 - e^{i eps~_mu T} <phi~_mu(0)| U_T |phi~_mu(0)>| with (phi~_mu,
      eps~_mu) the Floquet states of the step-h/2 chain and U_T the step-h chain: the overlap
      of one coarse period with the exact evolution e^{-i eps~ T} phi~ of the finer state.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.linalg import eigvalsh_tridiagonal
from scipy.special import jv


# ----------------------------------------------------------------------------- drive
def cos_drive(f_dc: float, f_ac: float, omega: float, phi0: float, t):
    """f, f', f'' of f(t) = f_dc + f_ac cos(omega t + phi0) (Eq. 13 with a cosine drive)."""
    arg = omega * np.asarray(t, dtype=np.float64) + phi0
    f = f_dc + f_ac * np.cos(arg)
    df = -f_ac * omega * np.sin(arg)
    d2f = -f_ac * omega * omega * np.cos(arg)
    return f, df, d2f


# ---------------------------------------------------------------------------- Magnus
def magnus4_coefficients(period: float, steps: int, f, df, d2f):
    """Per-step scalars of Omega_m = a_m H0 + b_m H1 + c_m i[H0,H1] (reading R1).

    Eq. 15: alpha_j = h^j/(j-1)! d^{j-1}A(t_1/2)/dt^{j-1}.  Eq. 14 truncated after the
    leading commutator gives Omega_A = alpha1 + alpha3/12 - [alpha1, alpha2]/12 for
    Y' = A Y.  With A = -iH, H = H0 + f H1 and Omega_H = i Omega_A:
        a_m = h,  b_m = h f(tau_m) + h^3 f''(tau_m)/24,  c_m = h^3 f'(tau_m)/12.
    `f`, `df`, `d2f` are callables of the midpoint times tau_m.
    """
    h = period / steps
    tau = (np.arange(steps, dtype=np.float64) + 0.5) * h
    a = np.full(steps, h)
    b = h * f(tau) + h ** 3 * d2f(tau) / 24.0
    c = h ** 3 * df(tau) / 12.0
    return h, a, b, c


GL3_NODES = (0.5 - math.sqrt(15.0) / 10.0, 0.5, 0.5 + math.sqrt(15.0) / 10.0)


def magnus6_from_alphas(a1, a2, a3):
    """Eq. 14 in full for Y' = A Y: C1 = [alpha1, alpha2], C2 = -(1/60)[alpha1, 2 alpha3 + C1],
    Omega_A = alpha1 + alpha3/12 + (1/240)[-20 alpha1 - alpha3 + C1, alpha2 + C2];
    returned as the Hermitian Omega_H = i Omega_A (U = exp(-i Omega_H))."""
    comm = lambda x, y: x @ y - y @ x
    c1 = comm(a1, a2)
    c2 = -comm(a1, 2.0 * a3 + c1) / 60.0
    return 1j * (a1 + a3 / 12.0 + comm(-20.0 * a1 - a3 + c1, a2 + c2) / 240.0)


def magnus6_omega_taylor(h0, h1, h, f, df, d2f):
    """Eq. 14 with the alphas of Eq. 15 taken literally as midpoint derivatives,
    alpha_j = h^j/(j-1)! A^(j-1)(t_1/2), A = -i(H0 + f H1).  Only 4th order for a general drive:
    alpha1 + alpha3/12 = h A + h^3 A^(2)/24 misses the h^5 A^(4)/1920 term of the integral of A."""
    a1 = -1j * h * (h0 + f * h1)
    a2 = -1j * h ** 2 * df * h1
    a3 = -1j * h ** 3 / 2.0 * d2f * h1
    return magnus6_from_alphas(a1, a2, a3)


def magnus6_omega(h0, h1, h, f1, f2, f3):
    """Reading R12: Eq. 14 with its alphas as the Gauss-Legendre moments of A = -i(H0 + f H1) at
    the nodes t + c_i h (c = 1/2 -+ sqrt(15)/10, 1/2), f_i = f(t + c_i h):
        alpha1 = h A_2, alpha2 = (sqrt(15) h / 3)(A_3 - A_1), alpha3 = (10 h / 3)(A_3 - 2 A_2 + A_1),
    which equal Eq. 15's derivative forms to leading order in h and make alpha1 + alpha3/12 the
    3-point Gauss quadrature of the integral of A, so the scheme is genuinely 6th order."""
    A1, A2, A3 = (-1j * (h0 + f * h1) for f in (f1, f2, f3))
    a1 = h * A2
    a2 = math.sqrt(15.0) * h / 3.0 * (A3 - A1)
    a3 = 10.0 * h / 3.0 * (A3 - 2.0 * A2 + A1)
    return magnus6_from_alphas(a1, a2, a3)


def plan_dense6(h0, h1, drive, steps, tol=1e-14):
    """Plan for the 6th-order scheme: per-step Omega_m/h kept explicitly; bounds are the extreme
    eigenvalues over all steps (exact LAPACK) plus the relative margin of 1e-12."""
    T = 2.0 * math.pi / drive.omega
    h = T / steps
    omegas = []
    lo, hi = np.inf, -np.inf
    for m in range(steps):
        fs = [float(cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, (m + c) * h)[0])
              for c in GL3_NODES]
        om = magnus6_omega(h0, h1, h, *fs)
        om = 0.5 * (om + om.conj().T)
        w = np.linalg.eigvalsh(om / h)
        lo, hi = min(lo, w[0]), max(hi, w[-1])
        omegas.append(om)
    plan = finish_plan(T, h, np.full(steps, h), np.zeros(steps), np.zeros(steps), lo, hi, 0.0, tol)
    return plan, omegas


def build_ut_dense6(plan, omegas):
    n = omegas[0].shape[0]
    x = np.eye(n, dtype=np.complex128)
    for om in omegas:
        omt = (om / plan.h - plan.beta * np.eye(n)) / plan.delta_e
        x = chebyshev_step(lambda v: omt @ v, x, plan.coeffs, plan.phase)
    return x


def piecewise_coefficients(period: float, fm):
    """Piecewise-constant amplitudes f_m: within a step H is constant, so f' = f'' = 0 and
    Eq. 14 reduces to Omega_m = h (H0 + f_m H1) exactly (a_m = h, b_m = h f_m, c_m = 0)."""
    fm = np.asarray(fm, dtype=np.float64)
    steps = fm.shape[0]
    h = period / steps
    return h, np.full(steps, h), h * fm, np.zeros(steps)


def commutator_dense(h0: np.ndarray, h1: np.ndarray) -> np.ndarray:
    """[H0, H1] = H0 H1 - H1 H0 (computed once, before the propagation; §3)."""
    return h0 @ h1 - h1 @ h0


def commutator_tridiag(h0_off: np.ndarray, h1_diag: np.ndarray) -> np.ndarray:
    """Lower off-diagonal of [H0, H1] for tridiagonal H0 and diagonal H1:
    [H0,H1]_{pq} = H0_{pq} (h1_q - h1_p); the diagonal vanishes and the upper
    off-diagonal is minus the lower one."""
    return h0_off * (h1_diag[:-1] - h1_diag[1:])


# ------------------------------------------------------------------ Chebyshev + Bessel
def chebyshev_order(R: float, tol: float = 1e-14, l_max: int = 100000) -> int:
    """Reading R5: L = smallest integer l > R, l >= 1, with |J_{l+1}(R)| < tol."""
    l = max(1, int(math.floor(R)) + 1)
    while l < l_max and abs(jv(l + 1, R)) >= tol:
        l += 1
    return l


def bessel_coefficients(R: float, L: int) -> np.ndarray:
    """Eq. 12: a_0 = J_0(R), a_l = 2 J_l(R), l = 1..L."""
    a = 2.0 * jv(np.arange(L + 1), R)
    a[0] *= 0.5
    return a


@dataclasses.dataclass
class Plan:
    """Everything the propagation needs besides the operators (host FP64)."""
    period: float
    steps: int
    h: float
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    e_min: float
    e_max: float
    beta: float
    delta_e: float
    R: float
    L: int
    coeffs: np.ndarray
    phase: complex


def finish_plan(period, h, a, b, c, lead_min, lead_max, comm_norm, tol) -> Plan:
    """Reading R4 (Weyl widening and margin) followed by Eqs. 11-12 (beta, Delta E, R, a_l)."""
    w = float(np.max(np.abs(c / h))) * comm_norm if len(c) else 0.0
    e_min, e_max = lead_min - w, lead_max + w
    margin = 1e-12 * max(abs(e_min), abs(e_max), 1.0)
    e_min, e_max = e_min - margin, e_max + margin
    delta_e = 0.5 * (e_max - e_min)
    beta = delta_e + e_min
    R = h * delta_e
    L = chebyshev_order(R, tol)
    return Plan(period, len(a), h, a, b, c, e_min, e_max, beta, delta_e, R, L,
                bessel_coefficients(R, L), complex(np.exp(-1j * beta * h)))


def _g_range(h, b, g_range):
    if g_range is not None:
        return float(g_range[0]), float(g_range[1])
    g = b / h
    return float(np.min(g)), float(np.max(g))


def frozen_g_range(fm) -> tuple[float, float]:
    """Reading R11: widen [min f, max f] by 10% of max(span, max|f|) on each side."""
    lo, hi = float(np.min(fm)), float(np.max(fm))
    pad = 0.1 * max(hi - lo, abs(lo), abs(hi), 1e-3)
    return lo - pad, hi + pad


def plan_dense(h0, h1, period, coeffs, tol=1e-14, g_range=None) -> Plan:
    """Spectral bounds of Omega_m/h by full diagonalisation at the extreme H1 coefficients
    (§3, "diagonalize ... and use the maximal and minimal values"; reading R4)."""
    h, a, b, c = coeffs
    g_lo, g_hi = _g_range(h, b, g_range)
    ev_lo = np.linalg.eigvalsh(h0 + g_lo * h1)
    ev_hi = np.linalg.eigvalsh(h0 + g_hi * h1)
    k = commutator_dense(h0, h1)
    comm_norm = float(np.max(np.abs(np.linalg.eigvalsh(1j * k)))) if np.any(c) else 0.0
    return finish_plan(period, h, a, b, c, min(ev_lo[0], ev_hi[0]),
                        max(ev_lo[-1], ev_hi[-1]), comm_norm, tol)


def _tridiag_extremes(diag, off):
    n = diag.shape[0]
    if n == 1:
        return float(diag[0]), float(diag[0])
    lo = eigvalsh_tridiagonal(diag, off, select="i", select_range=(0, 0))[0]
    hi = eigvalsh_tridiagonal(diag, off, select="i", select_range=(n - 1, n - 1))[0]
    return float(lo), float(hi)


def plan_tridiag(h0_diag, h0_off, h1_diag, period, coeffs, tol=1e-14, g_range=None) -> Plan:
    """Same bounds as plan_dense for tridiagonal H0 / diagonal H1 (tridiagonal eigensolver).
    ||[H0,H1]||_2: i[H0,H1] is Hermitian tridiagonal with zero diagonal, unitarily similar
    (diagonal phases) to the real tridiagonal matrix with off-diagonal |K_{i+1,i}|."""
    h, a, b, c = coeffs
    g_lo, g_hi = _g_range(h, b, g_range)
    lo1, hi1 = _tridiag_extremes(h0_diag + g_lo * h1_diag, h0_off)
    lo2, hi2 = _tridiag_extremes(h0_diag + g_hi * h1_diag, h0_off)
    comm_norm = 0.0
    if np.any(c) and h0_diag.shape[0] > 1:
        kl = np.abs(commutator_tridiag(h0_off, h1_diag))
        lo, hi = _tridiag_extremes(np.zeros_like(h0_diag), kl)
        comm_norm = max(abs(lo), abs(hi))
    return finish_plan(period, h, a, b, c, min(lo1, lo2), max(hi1, hi2), comm_norm, tol)


# ------------------------------------------------------------------ rescaled operator
def omega_tilde_dense(h0, h1, k, plan: Plan, m: int) -> np.ndarray:
    """Eq. 11 applied to Omega_m/h (reading R2): (Omega_m/h - beta 1)/Delta E, with
    Omega_m = a_m H0 + b_m H1 + c_m i[H0,H1] (reading R1).  m is 0-based."""
    n = h0.shape[0]
    omega = plan.a[m] * h0 + plan.b[m] * h1 + plan.c[m] * 1j * k
    return (omega / plan.h - plan.beta * np.eye(n)) / plan.delta_e


def omega_tilde_tridiag(h0_diag, h0_off, h1_diag, k_low, plan: Plan, m: int):
    """Tridiagonal form of omega_tilde_dense: returns (diag, lower) with
    Omega~[i,i] = diag[i] (real), Omega~[i+1,i] = lower[i], Omega~[i,i+1] = conj(lower[i])."""
    diag = ((plan.a[m] * h0_diag + plan.b[m] * h1_diag) / plan.h - plan.beta) / plan.delta_e
    lower = (plan.a[m] * h0_off + plan.c[m] * 1j * k_low) / plan.h / plan.delta_e
    return diag, lower


def apply_tridiag(diag, lower, x):
    """y = Omega~ x for the tridiagonal Hermitian Omega~ (x: n x c block of column states)."""
    y = diag[:, None] * x
    y[1:] += lower[:, None] * x[:-1]
    y[:-1] += np.conj(lower)[:, None] * x[1:]
    return y


def chebyshev_step(apply, x, coeffs, phase):
    """One propagation step, Eqs. 10 and 12:
    psi_0 = x, psi_1 = -i Omega~ psi_0, psi_{l+1} = -2i Omega~ psi_l + psi_{l-1},
    result = e^{-i beta h} sum_{l=0}^{L} a_l psi_l."""
    L = len(coeffs) - 1
    psi_prev = x
    psi = -1j * apply(psi_prev)
    acc = coeffs[0] * psi_prev + coeffs[1] * psi
    for l in range(1, L):
        psi_next = -2j * apply(psi) + psi_prev
        acc = acc + coeffs[l + 1] * psi_next
        psi_prev, psi = psi, psi_next
    return phase * acc


# ------------------------------------------------------------------------ propagation
def propagate_dense(h0, h1, plan: Plan, x0, m_begin=0, m_end=None):
    """Chain of Eq. 9 from step m_begin to m_end (0-based, exclusive end) on the block x0
    (n x c, one state per column); the step loop of Algorithm 1."""
    m_end = plan.steps if m_end is None else m_end
    k = commutator_dense(h0, h1)
    x = np.array(x0, dtype=np.complex128)
    for m in range(m_begin, m_end):
        om = omega_tilde_dense(h0, h1, k, plan, m)
        x = chebyshev_step(lambda v: om @ v, x, plan.coeffs, plan.phase)
    return x


def propagate_tridiag(h0_diag, h0_off, h1_diag, plan: Plan, x0, m_begin=0, m_end=None):
    """As propagate_dense with the tridiagonal Omega~."""
    m_end = plan.steps if m_end is None else m_end
    k_low = commutator_tridiag(h0_off, h1_diag)
    x = np.array(x0, dtype=np.complex128)
    for m in range(m_begin, m_end):
        d, lo = omega_tilde_tridiag(h0_diag, h0_off, h1_diag, k_low, plan, m)
        x = chebyshev_step(lambda v: apply_tridiag(d, lo, v), x, plan.coeffs, plan.phase)
    return x


def build_ut_dense(h0, h1, plan: Plan):
    """U_T: propagation of the n x n identity over one period (§3, last paragraph)."""
    return propagate_dense(h0, h1, plan, np.eye(h0.shape[0]))


def build_ut_tridiag(h0_diag, h0_off, h1_diag, plan: Plan, columns=None):
    """U_T (or the listed columns of it): each column is basis vector e_j propagated
    independently (§5, Fig. 2: the columns do not interact)."""
    n = h0_diag.shape[0]
    cols = np.arange(n) if columns is None else np.asarray(columns)
    x0 = np.zeros((n, len(cols)), dtype=np.complex128)
    x0[cols, np.arange(len(cols))] = 1.0
    return propagate_tridiag(h0_diag, h0_off, h1_diag, plan, x0)


# --------------------------------------------------------------- convenience wrappers
def plan_for_drive_dense(h0, h1, drive, steps, tol=1e-14):
    T = 2.0 * math.pi / drive.omega
    f = lambda t: cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[0]
    df = lambda t: cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[1]
    d2f = lambda t: cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[2]
    return plan_dense(h0, h1, T, magnus4_coefficients(T, steps, f, df, d2f), tol)


def plan_for_drive_tridiag(h0_diag, h0_off, h1_diag, drive, steps, tol=1e-14):
    T = 2.0 * math.pi / drive.omega
    f = lambda t: cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[0]
    df = lambda t: cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[1]
    d2f = lambda t: cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[2]
    return plan_tridiag(h0_diag, h0_off, h1_diag, T,
                        magnus4_coefficients(T, steps, f, df, d2f), tol)


# ------------------------------------------------------------------ outputs of U_T
def quasienergies(u: np.ndarray, period: float) -> np.ndarray:
    """Eqs. 4-5 with reading R7: U_T phi = e^{-i theta} phi, eps = theta/T,
    theta = -arg(lambda) in [-pi, pi); returned sorted ascending.  Eigenvalues by
    LAPACK zgeev (§5; the last part of Algorithm 1)."""
    lam = np.linalg.eigvals(u)
    theta = -np.angle(lam)
    theta = np.where(theta >= math.pi, theta - 2.0 * math.pi, theta)
    return np.sort(theta / period)


def overlap_phase_error(u_coarse: np.ndarray, u_fine: np.ndarray, period: float):
    """Eq. 20 with reading R14.  Returns (eps~ ascending, Sigma_mu in that order); the Floquet
    states of u_fine come from LAPACK zgeev, normalised."""
    lam, v = np.linalg.eig(u_fine)
    theta = -np.angle(lam)
    theta = np.where(theta >= math.pi, theta - 2.0 * math.pi, theta)
    order = np.argsort(theta)
    theta = theta[order]
    v = v[:, order]
    v = v / np.linalg.norm(v, axis=0, keepdims=True)
    sigma = np.empty(len(theta))
    for mu in range(len(theta)):
        phi = v[:, mu]
        overlap = np.vdot(phi, u_coarse @ phi)
        sigma[mu] = abs(1.0 - np.exp(1j * theta[mu]) * overlap)
    return theta / period, sigma


def simpson_weights(steps: int, h: float) -> np.ndarray:
    """Quadrature weights over the step boundaries t_m = m h, m = 0..M: composite Simpson for
    even M, trapezoid for odd M."""
    w = np.full(steps + 1, h)
    if steps % 2 == 0:
        w[1:-1:2] = 4.0 * h / 3.0
        w[2:-1:2] = 2.0 * h / 3.0
        w[0] = w[-1] = h / 3.0
    else:
        w[0] = w[-1] = h / 2.0
    return w


def average_observable(propagate_step, expect, x0, drive, steps):
    """Eq. 17: <A>_T = (1/T) int_0^T <psi(t)|A(t)|psi(t)> dt for each column state of x0,
    evaluated at the step boundaries of the chain (second propagation round of §3).
    `propagate_step(m, x)` applies step m, `expect(t, x)` returns <x_c|A(t)|x_c> per column."""
    T = 2.0 * math.pi / drive.omega
    h = T / steps
    w = simpson_weights(steps, h)
    x = np.array(x0, dtype=np.complex128)
    acc = w[0] * expect(0.0, x)
    for m in range(steps):
        x = propagate_step(m, x)
        acc = acc + w[m + 1] * expect((m + 1) * h, x)
    return acc / T


def expect_dense(h0, h1, a0, a1, s_drive, drive):
    """<x|A(t)|x> per column with A(t) = a0 H0 + (a1 + s_drive f(t)) H1 (dense)."""
    def ev(t, x):
        f = float(cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[0])
        a = a0 * h0 + (a1 + s_drive * f) * h1
        return np.real(np.einsum("ic,ic->c", np.conj(x), a @ x))
    return ev


def expect_tridiag(h0_diag, h0_off, h1_diag, a0, a1, s_drive, drive):
    """expect_dense for tridiagonal H0 (diagonal, off-diagonal) and diagonal H1: <x|A(t)|x> per
    column with A(t) = a0 H0 + (a1 + s_drive f(t)) H1, the integrand of Eq. 17 for the dimer."""
    def ev(t, x):
        f = float(cos_drive(drive.f_dc, drive.f_ac, drive.omega, drive.phi0, t)[0])
        d = a0 * h0_diag + (a1 + s_drive * f) * h1_diag
        y = apply_tridiag(d, (a0 * h0_off).astype(np.complex128), x)
        return np.real(np.einsum("ic,ic->c", np.conj(x), y))
    return ev


def unitarity_defect(u: np.ndarray) -> tuple[float, float]:
    """max |U^+ U - 1| and ||U^+ U - 1||_F / sqrt(n) (unitarity of Eq. 9, §2)."""
    d = u.conj().T @ u - np.eye(u.shape[0])
    return float(np.max(np.abs(d))), float(np.linalg.norm(d) / math.sqrt(u.shape[0]))


# ------------------------------------------------------------- gate-fidelity adjoint
def fidelity_loss(u: np.ndarray, target: np.ndarray) -> tuple[float, complex]:
    """L = 1 - |Tr(W^+ U_T)|^2 / N^2; returns (L, tau = Tr(W^+ U_T))."""
    n = u.shape[0]
    tau = complex(np.sum(np.conj(target) * u))
    return 1.0 - abs(tau) ** 2 / n ** 2, tau


def plan_piecewise(h0, h1, period, fm, tol=1e-14, g_range=None) -> Plan:
    """Plan for piecewise-constant amplitudes with frozen bounds (reading R11)."""
    coeffs = piecewise_coefficients(period, fm)
    return plan_dense(h0, h1, period, coeffs, tol,
                      g_range if g_range is not None else frozen_g_range(fm))


def forward_piecewise(h0, h1, plan: Plan, fm):
    """U_T for amplitudes fm under a frozen plan: Omega~_m = (H0 + f_m H1 - beta)/Delta E."""
    n = h0.shape[0]
    x = np.eye(n, dtype=np.complex128)
    for m in range(len(fm)):
        om = (h0 + fm[m] * h1 - plan.beta * np.eye(n)) / plan.delta_e
        x = chebyshev_step(lambda v: om @ v, x, plan.coeffs, plan.phase)
    return x


def loss_piecewise(h0, h1, target, plan: Plan, fm) -> float:
    return fidelity_loss(forward_piecewise(h0, h1, plan, fm), target)[0]


def grad_piecewise(h0, h1, target, plan: Plan, fm):
    """Discrete adjoint of the Magnus-Chebyshev chain (reverse mode through Eqs. 9, 10, 12).

    Convention dL = 2 Re <G, dU>, <A, B> = Tr(A^+ B); seed G_M = -tau W / N^2.
    For step m (descending) with X_{m-1} its input and psi_l its Chebyshev vectors:
      bbar_l = conj(e^{-i beta h}) a_l G_m + conj(w_{l+1}) Omega~ bbar_{l+1} + bbar_{l+2}
      (bbar_{L+1} = bbar_{L+2} = 0, w_1 = -i, w_l = -2i for l >= 2),
      dL/df_m = 2 Re sum_{l=1}^{L} <bbar_l, w_l E psi_{l-1}>,  E = dOmega~/df_m = H1/Delta E,
      G_{m-1} = bbar_0 (= U_m^+ G_m).
    Plain loops; every X_m is kept (no checkpointing)."""
    n = h0.shape[0]
    steps = len(fm)
    L = plan.L
    a = plan.coeffs
    eye = np.eye(n)
    xs = [np.eye(n, dtype=np.complex128)]
    for m in range(steps):
        om = (h0 + fm[m] * h1 - plan.beta * eye) / plan.delta_e
        xs.append(chebyshev_step(lambda v: om @ v, xs[-1], a, plan.phase))
    loss, tau = fidelity_loss(xs[-1], target)
    g = -tau * target / n ** 2
    e = h1 / plan.delta_e
    w = [0j, -1j] + [-2j] * (L - 1)
    grad = np.zeros(steps)
    for m in range(steps - 1, -1, -1):
        om = (h0 + fm[m] * h1 - plan.beta * eye) / plan.delta_e
        psi = [xs[m], -1j * (om @ xs[m])]
        for l in range(1, L):
            psi.append(-2j * (om @ psi[l]) + psi[l - 1])
        bbar = [None] * (L + 3)
        zero = np.zeros((n, n), dtype=np.complex128)
        bbar[L + 1] = zero
        bbar[L + 2] = zero
        for l in range(L, -1, -1):
            v = np.conj(plan.phase) * a[l] * g + bbar[l + 2]
            if l + 1 <= L:
                v = v + np.conj(w[l + 1]) * (om @ bbar[l + 1])
            bbar[l] = v
        s = 0.0
        for l in range(1, L + 1):
            s += 2.0 * float(np.real(np.vdot(bbar[l], w[l] * (e @ psi[l - 1]))))
        grad[m] = s
        g = bbar[0]
    return loss, grad

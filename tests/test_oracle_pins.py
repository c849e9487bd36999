"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test ties one part of the oracle to something other than the oracle itself:
closed forms, textbook integrators, exact identities and invariants.  Each is chosen so
that a plausible slip (a dropped term, a wrong sign, a transposed operand, the wrong
product order) fails it.
"""
import math

import numpy as np
import pytest
from scipy.special import jv

import floquet_inputs as fi
import oracle as o


# ------------------------------------------------------------------ helpers (tests only)
def expm_herm(h: np.ndarray, t: float) -> np.ndarray:
    """exp(-i t H) for Hermitian H via its eigendecomposition (library eigh)."""
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-1j * t * w)[None, :]) @ v.conj().T


def rk4_propagator(h0, h1, drive, t_end, nsteps):
    """Classical 4th-order Runge-Kutta for i U' = H(t) U, U(0) = 1 (textbook integrator)."""
    n = h0.shape[0]
    u = np.eye(n, dtype=np.complex128)
    k = t_end / nsteps

    def rhs(t, y):
        f = drive.f_dc + drive.f_ac * math.cos(drive.omega * t + drive.phi0)
        return -1j * ((h0 + f * h1) @ y)

    t = 0.0
    for _ in range(nsteps):
        k1 = rhs(t, u)
        k2 = rhs(t + k / 2, u + k / 2 * k1)
        k3 = rhs(t + k / 2, u + k / 2 * k2)
        k4 = rhs(t + k, u + k * k3)
        u = u + k / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += k
    return u


# ------------------------------------------------------------------------ Bessel / L
@pytest.mark.parametrize("R", [1e-3, 0.0859, 0.5, 1.0, 13.947, 40.0])
def test_bessel_jacobi_anger(R):
    """Eq. 12 coefficients reproduce e^{-iRx} = sum_l a_l (-i)^l T_l(x) on [-1, 1]
    (Jacobi-Anger expansion; T_l(cos th) = cos(l th))."""
    L = o.chebyshev_order(R, 1e-14)
    a = o.bessel_coefficients(R, L)
    th = np.linspace(0.0, math.pi, 37)
    ls = np.arange(L + 1)
    series = ((-1j) ** ls[None, :] * a[None, :] * np.cos(np.outer(th, ls))).sum(axis=1)
    exact = np.exp(-1j * R * np.cos(th))
    assert np.max(np.abs(series - exact)) < 5e-14 * (1.0 + R)
    # reading R5: L > R and |J_{L+1}| < tol, and L is the first such index
    assert L > R and abs(jv(L + 1, R)) < 1e-14
    assert L == max(1, math.floor(R) + 1) or abs(jv(L, R)) >= 1e-14


def test_bessel_sum_rule():
    """J_0(R) + 2 sum_k J_{2k}(R) = 1 (generating function at t = 1)."""
    for R in (0.1, 3.0, 13.947):
        L = o.chebyshev_order(R)
        a = o.bessel_coefficients(R, L)
        assert abs(a[0] + a[2::2].sum() - 1.0) < 1e-14


# ------------------------------------------------------------------- one step
def test_chebyshev_step_matches_exponential():
    """One step of Eqs. 10-12 equals exp(-i h Omega/h) built from the eigendecomposition."""
    n = 12
    hmat = fi.goe(n, 101) + 0.3 * fi.goe(n, 102) * 1j
    hmat = 0.5 * (hmat + hmat.conj().T)
    h = 0.37
    w = np.linalg.eigvalsh(hmat)
    plan = o.finish_plan(h, h, np.array([h]), np.array([0.0]), np.array([0.0]),
                          w[0], w[-1], 0.0, 1e-14)
    omt = (hmat - plan.beta * np.eye(n)) / plan.delta_e
    x0 = fi.ginibre(n, 103)[:, :5]
    got = o.chebyshev_step(lambda v: omt @ v, x0, plan.coeffs, plan.phase)
    want = expm_herm(hmat, h) @ x0
    assert np.max(np.abs(got - want)) < 1e-13


# ------------------------------------------------------------------- Magnus pieces
def test_magnus_coefficients_against_integrals():
    """b_m -> integral of f over the step and c_m -> the exact scalar of the second Magnus
    term, -(1/2) int_{t0}^{t1} ds int_{t0}^{s} ds' (f(s') - f(s)) (Eq. 8 with
    [H(s), H(s')] = (f(s') - f(s)) [H0, H1]); both per-step errors are O(h^5), so they fall
    by ~2^5 when M doubles, and agree in sign and size already at M = 40."""
    drv = fi.Drive(0.4, 1.3, 1.7, 0.9)
    T = drv.period
    F = lambda t: drv.f_dc * t + drv.f_ac / drv.omega * np.sin(drv.omega * t + drv.phi0)
    f = lambda t: drv.f_dc + drv.f_ac * np.cos(drv.omega * t + drv.phi0)
    xg, wg = np.polynomial.legendre.leggauss(30)
    errs_b, errs_c = [], []
    for M in (40, 80):
        h, a, b, c = o.magnus4_coefficients(
            T, M, *[lambda t, k=k: o.cos_drive(drv.f_dc, drv.f_ac, drv.omega, drv.phi0, t)[k]
                    for k in range(3)])
        assert np.allclose(a, h)
        t0 = np.arange(M) * h
        eb = np.abs(b - (F(t0 + h) - F(t0)))
        c_exact = np.zeros(M)
        for m in range(M):
            s1 = t0[m] + (xg + 1) * h / 2
            tot = 0.0
            for si, wi in zip(s1, wg):
                s2 = t0[m] + (xg + 1) * (si - t0[m]) / 2
                tot += wi * h / 2 * np.sum(wg * (si - t0[m]) / 2 * (f(s2) - f(si)))
            c_exact[m] = -0.5 * tot
        ec = np.abs(c - c_exact)
        assert np.max(ec) < 2e-3 * np.max(np.abs(c_exact))
        errs_b.append(eb.max())
        errs_c.append(ec.max())
    assert errs_b[0] / errs_b[1] > 25.0 and errs_c[0] / errs_c[1] > 25.0, (errs_b, errs_c)


def test_commuting_pair_closed_form():
    """[H0, H1] = 0: the chain is exp(-i(T H0 + sum_m b_m H1)) and, over a full period of a
    cosine drive, sum_m b_m = f_dc T exactly, so U_T = exp(-i T (H0 + f_dc H1))."""
    n = 10
    h0 = fi.goe(n, 201)
    h1 = h0 @ h0 - 0.3 * h0
    drv = fi.Drive(0.7, 1.1, 1.3, 0.25)
    plan = o.plan_for_drive_dense(h0, h1, drv, 24)
    got = o.build_ut_dense(h0, h1, plan)
    want = expm_herm(h0 + drv.f_dc * h1, drv.period)
    assert np.max(np.abs(got - want)) < 1e-12


def test_undriven_limit():
    """f = 0: U_T = exp(-i H0 T) (eigendecomposition), the undriven check of the method."""
    h0 = fi.goe(32, 301)
    h1 = fi.goe(32, 302)
    drv = fi.Drive(0.0, 0.0, 1.0)
    plan = o.plan_for_drive_dense(h0, h1, drv, 50)
    got = o.build_ut_dense(h0, h1, plan)
    assert np.max(np.abs(got - expm_herm(h0, drv.period))) < 1e-12


def _errors_vs_rk4(c_sign=1.0):
    h0, h1 = fi.goe(4, 11), fi.goe(4, 12)
    drv = fi.Drive(0.3, 1.2, 1.3, 0.7)          # not even about T/2: pins the product order
    ref = rk4_propagator(h0, h1, drv, drv.period, 1 << 13)
    errs = []
    for M in (16, 32, 64):
        plan = o.plan_for_drive_dense(h0, h1, drv, M)
        plan.c = c_sign * plan.c
        errs.append(np.max(np.abs(o.build_ut_dense(h0, h1, plan) - ref)))
    return errs


def test_fourth_order_convergence_against_rk4():
    """Global error of the Magnus-4 chain against an independent RK4 solution falls by
    ~2^4 per doubling of M (and the chain converges to it: right order of the product)."""
    e = _errors_vs_rk4()
    assert e[0] < 5e-2
    for r in (e[0] / e[1], e[1] / e[2]):
        assert 12.0 < r < 20.0, e


def test_order_test_catches_commutator_sign():
    """Planted mistake (in the oracle, on the CPU): flipping the sign of c_m must drop the
    observed order to ~2, so the convergence test above really pins c_m."""
    e = _errors_vs_rk4(-1.0)
    assert e[1] / e[2] < 6.0


def test_sixth_order_convergence_against_rk4():
    """The full Eq. 14 (6th order, nine commutators) converges as h^6: error ratio ~2^6 per
    doubling of M against the independent RK4 solution (non-even drive)."""
    h0, h1 = fi.goe(4, 11), fi.goe(4, 12)
    drv = fi.Drive(0.3, 1.2, 1.3, 0.7)
    ref = rk4_propagator(h0, h1, drv, drv.period, 1 << 14)
    errs = []
    for M in (8, 16, 32):
        plan, oms = o.plan_dense6(h0, h1, drv, M)
        errs.append(np.max(np.abs(o.build_ut_dense6(plan, oms) - ref)))
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 50.0 < r < 80.0, errs


def test_sixth_order_literal_derivative_alphas_are_fourth_order():
    """Reading R12 is needed: Eq. 14 with Eq. 15's alphas taken literally as midpoint derivatives
    converges only as h^4 (ratio ~16), because alpha1 + alpha3/12 misses the h^5 term of the
    integral of A; and for a constant drive both forms reduce to h (H0 + f H1) exactly."""
    h0, h1 = fi.goe(4, 11), fi.goe(4, 12)
    drv = fi.Drive(0.3, 1.2, 1.3, 0.7)
    ref = rk4_propagator(h0, h1, drv, drv.period, 1 << 14)
    errs = []
    for M in (16, 32):
        h = drv.period / M
        u = np.eye(4, dtype=complex)
        for m in range(M):
            f, df, d2f = (float(v) for v in o.cos_drive(drv.f_dc, drv.f_ac, drv.omega, drv.phi0, (m + 0.5) * h))
            om = o.magnus6_omega_taylor(h0, h1, h, f, df, d2f)
            u = expm_herm(0.5 * (om + om.conj().T), 1.0) @ u
        errs.append(np.max(np.abs(u - ref)))
    assert 12.0 < errs[0] / errs[1] < 20.0, errs
    h0, h1 = fi.goe(5, 21), fi.goe(5, 22)
    h, f = 0.1, 0.7
    assert np.max(np.abs(o.magnus6_omega(h0, h1, h, f, f, f) - h * (h0 + f * h1))) < 1e-14
    assert np.max(np.abs(o.magnus6_omega_taylor(h0, h1, h, f, 0.0, 0.0) - h * (h0 + f * h1))) < 1e-14


def test_bounds_contain_every_step_spectrum():
    """Reading R4: [E_min, E_max] contains the spectrum of Omega_m/h at every step."""
    h0, h1 = fi.goe(16, 401), fi.goe(16, 402)
    drv = fi.Drive(0.2, 1.5, 0.8, 0.3)
    plan = o.plan_for_drive_dense(h0, h1, drv, 12)
    k = o.commutator_dense(h0, h1)
    for m in range(12):
        w = np.linalg.eigvalsh((plan.a[m] * h0 + plan.b[m] * h1 + plan.c[m] * 1j * k) / plan.h)
        assert plan.e_min <= w[0] and w[-1] <= plan.e_max


# -------------------------------------------------------------------- invariants
def test_unitarity_and_even_drive_symmetry():
    """U_T is unitary to round-off (§2), and for real-symmetric H0, H1 with a drive even
    about T/2, Omega_{M+1-m} = Omega_m^T so U_T = U_T^T exactly; a phase offset breaks it."""
    m = fi.config_goe64()
    plan = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    u = o.build_ut_dense(m.h0, m.h1, plan)
    dmax, dfro = o.unitarity_defect(u)
    assert dmax < 1e-12 and dfro < 1e-12
    assert np.max(np.abs(u - u.T)) < 1e-13
    h0, h1 = fi.goe(16, 501), fi.goe(16, 502)
    u2 = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, fi.Drive(0, 1, 1, 0.6), 40))
    assert np.max(np.abs(u2 - u2.T)) > 1e-3


def test_quasienergies_undriven_fold():
    """Undriven: quasienergies are the eigenvalues of H0 folded into [-omega/2, omega/2)."""
    h0 = 3.0 * fi.goe(20, 601)
    drv = fi.Drive(0.0, 0.0, 2.0)
    plan = o.plan_for_drive_dense(h0, fi.goe(20, 602), drv, 30)
    eps = o.quasienergies(o.build_ut_dense(h0, 0 * h0, plan), drv.period)
    E = np.linalg.eigvalsh(h0)
    folded = np.sort((E + drv.omega / 2) % drv.omega - drv.omega / 2)
    assert np.all(eps >= -drv.omega / 2) and np.all(eps < drv.omega / 2)
    assert np.max(np.abs(eps - folded)) < 1e-10


# -------------------------------------------------------------------- dimer
def _su2_exp(w0, wx, wy, wz, t=1.0):
    """exp(-i t (w0 + w.sigma)) in closed form."""
    r = math.sqrt(wx * wx + wy * wy + wz * wz)
    c, s = math.cos(t * r), (math.sin(t * r) / r if r > 0 else t)
    sx = np.array([[0, 1], [1, 0]], complex)
    sy = np.array([[0, -1j], [1j, 0]])
    sz = np.array([[1, 0], [0, -1]], complex)
    return np.exp(-1j * t * w0) * (c * np.eye(2) - 1j * s * (wx * sx + wy * sy + wz * sz))


def _spin_rep(u, nb):
    """Fock-space image D(u) of a 2x2 mode transformation a_k^+ -> sum_l u_lk a_l^+ on the
    nb-boson basis |n, nb-n> (n bosons in mode 1)."""
    from math import comb, factorial
    D = np.zeros((nb + 1, nb + 1), complex)
    for n in range(nb + 1):
        norm_in = math.sqrt(factorial(n) * factorial(nb - n))
        for p in range(n + 1):
            for q in range(nb - n + 1):
                k = p + q
                coef = (comb(n, p) * comb(nb - n, q) * u[0, 0] ** p * u[1, 0] ** (n - p)
                        * u[0, 1] ** q * u[1, 1] ** (nb - n - q))
                D[k, n] += coef * math.sqrt(factorial(k) * factorial(nb - k)) / norm_in
    return D


def test_dimer_u0_is_spin_representation():
    """U = 0 dimer: H = -2J J_x + f J_z is the nb-boson image of h = [[f/2, -J], [-J, -f/2]];
    commutators map to commutators, so the Magnus chain equals D(u) with u the 2x2 chain of
    exact exponentials exp(-i(a h0 + b h1 + c i[h0, h1])) (closed form), and
    Tr U_T = sum_k l1^k l2^(nb-k) (character)."""
    nb, J = 24, 1.0
    d, off, h1d = fi.dimer_matrices(nb, J, U=0.0)
    drv = fi.Drive(0.2, 1.5, 3.0, 0.4)
    M = 48
    plan = o.plan_for_drive_tridiag(d, off, h1d, drv, M)
    got = o.build_ut_tridiag(d, off, h1d, plan)
    # 2x2 chain: h0 = -J sigma_x, h1 = sigma_z / 2, i[h0, h1] = -J sigma_y
    u = np.eye(2, dtype=complex)
    for m in range(M):
        wx = -J * plan.a[m]
        wz = 0.5 * plan.b[m]
        wy = -J * plan.c[m]
        u = _su2_exp(0.0, wx, wy, wz) @ u
    want = _spin_rep(u, nb)
    assert np.max(np.abs(got - want)) < 1e-11
    l1, l2 = np.linalg.eigvals(u)
    char = sum(l1 ** k * l2 ** (nb - k) for k in range(nb + 1))
    assert abs(np.trace(got) - char) < 1e-10


def test_paper_dimer_u0_is_spin_representation():
    """The paper's dimer form at U = 0: H0 = -v(a1^+ a2 + h.c.) = -2v J_x and H_mod = n2 - n1 =
    -2 J_z, the nb-boson image of h0 = -v sigma_x, h1 = -sigma_z (i[h0, h1] = 2v sigma_y), with
    the paper's dc + ac drive; U_T = D(u) for the 2x2 chain of exact exponentials."""
    nb, v = 20, 1.0
    d, off, h1d = fi.dimer_matrices_paper(nb, v, U=0.0)
    drv = fi.Drive(2.7, 2.5, 3.0)
    M = 400
    plan = o.plan_for_drive_tridiag(d, off, h1d, drv, M)
    got = o.build_ut_tridiag(d, off, h1d, plan)
    u = np.eye(2, dtype=complex)
    for m in range(M):
        u = _su2_exp(0.0, -v * plan.a[m], 2 * v * plan.c[m], -plan.b[m]) @ u
    assert np.max(np.abs(got - _spin_rep(u, nb))) < 1e-10


def test_tridiagonal_form_matches_dense_form():
    """The tridiagonal operator path (diag/lower, commutator by formula) agrees with the
    dense path on the same dimer written as full matrices (transposition/conjugation pin)."""
    nb = 30
    d, off, h1d = fi.dimer_matrices(nb, 1.0, U=0.07)
    drv = fi.Drive(0.3, 1.5, 3.0, 0.5)
    M = 20
    pt = o.plan_for_drive_tridiag(d, off, h1d, drv, M)
    ut = o.build_ut_tridiag(d, off, h1d, pt)
    h0 = np.diag(d) + np.diag(off, -1) + np.diag(off, 1)
    h1 = np.diag(h1d)
    pd = o.plan_for_drive_dense(h0, h1, drv, M)
    ud = o.build_ut_dense(h0, h1, pd)
    assert abs(pt.e_min - pd.e_min) < 1e-9 and abs(pt.e_max - pd.e_max) < 1e-9
    assert np.max(np.abs(ut - ud)) < 1e-11
    cols = [0, 7, 30]
    assert np.max(np.abs(o.build_ut_tridiag(d, off, h1d, pt, cols) - ut[:, cols])) < 1e-14


# -------------------------------------------------------------------- adjoint
def test_adjoint_matches_central_differences():
    """Discrete adjoint of the chain vs central finite differences of the same frozen-plan
    forward map (FP64, relative agreement <= 1e-6)."""
    n, M = 6, 10
    h0, h1 = fi.goe(n, 701), fi.goe(n, 702)
    w = fi.haar_unitary(n, 703)
    fm = 1.0 + 0.1 * fi.normal(704, M)
    plan = o.plan_piecewise(h0, h1, 2 * math.pi, fm)
    loss, grad = o.grad_piecewise(h0, h1, w, plan, fm)
    assert abs(loss - o.loss_piecewise(h0, h1, w, plan, fm)) < 1e-14
    for m in range(M):
        d = 1e-5 * abs(fm[m])
        fp, fmn = fm.copy(), fm.copy()
        fp[m] += d
        fmn[m] -= d
        fd = (o.loss_piecewise(h0, h1, w, plan, fp) - o.loss_piecewise(h0, h1, w, plan, fmn)) / (2 * d)
        assert abs(fd - grad[m]) <= 1e-6 * max(abs(grad).max(), 1e-12)
    v = fi.normal(705, M)
    dd = 1e-5
    fd = (o.loss_piecewise(h0, h1, w, plan, fm + dd * v)
          - o.loss_piecewise(h0, h1, w, plan, fm - dd * v)) / (2 * dd)
    assert abs(fd - grad @ v) <= 1e-6 * abs(grad @ v)


# -------------------------------------------------------------------- golden anchors
@pytest.mark.parametrize("name", ["goe64", "dimer40"])
def test_golden_regression(name):
    """The oracle reproduces its stored anchors (written by tests/golden/make_golden.py)."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    plan, u, eps = getattr(mg, name)()
    g = mg.read(name + ".txt")
    assert plan.L == int(g["L"]) and abs(plan.R - g["R"]) < 1e-12 * max(1.0, g["R"])
    assert np.max(np.abs(eps - np.array(g["eps"]))) < 1e-11
    for i, j, v in g["u"]:
        assert abs(u[i, j] - v) < 1e-12


# -------------------------------------------------------------- period averages (Eq. 17)
def test_average_energy_of_stationary_states():
    """Undriven: eigenvectors of H0 are stationary, so <H(t)>_T equals their eigenvalues."""
    n, M = 8, 40
    h0, h1 = fi.goe(n, 41), fi.goe(n, 42)
    drv = fi.Drive(0.0, 0.0, 1.7)
    E, V = np.linalg.eigh(h0)
    p = o.plan_for_drive_dense(h0, h1, drv, M)
    k = o.commutator_dense(h0, h1)
    step = lambda m, x: o.chebyshev_step(lambda v: o.omega_tilde_dense(h0, h1, k, p, m) @ v, x, p.coeffs, p.phase)
    avg = o.average_observable(step, o.expect_dense(h0, h1, 1.0, 0.0, 1.0, drv), V, drv, M)
    assert np.max(np.abs(avg - E)) < 1e-12


def test_average_h1_is_quasienergy_slope():
    """Floquet Hellmann-Feynman: for H = H0 + (f_dc + f_ac cos wt) H1, d eps_mu / d f_dc equals the
    period average <H1>_T of Floquet state mu (Eq. 17 with A = H1): a relation between the
    quasienergies (eigenvalues of U_T) and the second propagation round."""
    n, M = 6, 80
    h0, h1 = fi.goe(n, 31), fi.goe(n, 32)

    def quasi(fdc):
        drv = fi.Drive(fdc, 0.9, 1.3, 0.0)
        p = o.plan_for_drive_dense(h0, h1, drv, M)
        lam, V = np.linalg.eig(o.build_ut_dense(h0, h1, p))
        return lam, V, drv, p

    fdc, d = 0.2, 1e-4
    lam, V, drv, p = quasi(fdc)
    match = lambda l0, l1: np.array([l1[np.argmin(np.abs(l1 - x))] for x in l0])
    lp, lm = quasi(fdc + d)[0], quasi(fdc - d)[0]
    slope = (-np.angle(match(lam, lp) / lam) + np.angle(match(lam, lm) / lam)) / (2 * d * drv.period)
    k = o.commutator_dense(h0, h1)
    step = lambda m, x: o.chebyshev_step(lambda v: o.omega_tilde_dense(h0, h1, k, p, m) @ v, x, p.coeffs, p.phase)
    avg = o.average_observable(step, o.expect_dense(h0, h1, 0.0, 1.0, 0.0, drv), V / np.linalg.norm(V, axis=0),
                               drv, M)
    assert np.max(np.abs(slope - avg)) < 1e-6


# -------------------------------------------------------------------- overlap phase error (Eq. 20)
def test_overlap_phase_error_undriven_is_truncation_level():
    """With f = const the Magnus exponent is exact and both chains equal exp(-i H T) up to the
    Chebyshev truncation, so Sigma_mu vanishes to rounding; a wrong sign of the quasienergy
    phase would give |1 - e^{2 i eps T}| = O(1)."""
    h0, h1 = fi.goe(12, 1601), fi.goe(12, 1602)
    drv = fi.Drive(0.4, 0.0, 1.0)
    uc = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, 10))
    uf = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, 20))
    eps, sig = o.overlap_phase_error(uc, uf, drv.period)
    assert np.max(sig) < 1e-12
    assert np.all(np.diff(eps) >= 0)


def test_overlap_phase_error_decays_at_fourth_order():
    """Driven GOE: the one-period error of the 4th-order chain is O(h^4), so Sigma(M) against
    the 2M chain drops by about 2^4 per doubling of M (finer reference error included)."""
    h0, h1 = fi.goe(10, 1701), fi.goe(10, 1702)
    drv = fi.Drive(0.2, 1.2, 1.3, 0.4)
    u = {M: o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M)) for M in (16, 32, 64, 128)}
    s = [np.max(o.overlap_phase_error(u[M], u[2 * M], drv.period)[1]) for M in (16, 32, 64)]
    for a, b in zip(s, s[1:]):
        assert 12.0 < a / b < 20.0, s


def test_expect_tridiag_matches_dense_form():
    """<x|A(t)|x> of the tridiagonal form (Eq. 17's integrand for the dimer) against the dense
    form on the same dimer written as full matrices: driven, with a0, a1 and s all non-zero and
    different and a phase offset, at several instants and on complex states.  A swapped a0 / a1,
    a dropped off-diagonal or a wrong drive factor changes the result at O(1)."""
    nb = 24
    d, off, h1d = fi.dimer_matrices(nb, 1.0, U=0.11)
    h0 = np.diag(d) + np.diag(off, -1) + np.diag(off, 1)
    h1 = np.diag(h1d).astype(np.float64)
    drv = fi.Drive(0.35, 1.4, 2.3, 0.6)
    a0, a1, s = 0.7, -1.3, 2.1
    rng = np.random.default_rng(5)
    x = rng.standard_normal((nb + 1, 5)) + 1j * rng.standard_normal((nb + 1, 5))
    et = o.expect_tridiag(d, off, h1d, a0, a1, s, drv)
    ed = o.expect_dense(h0, h1, a0, a1, s, drv)
    for t in (0.0, 0.37, 1.9, drv.period * 0.8):
        got, ref = et(t, x), ed(t, x)
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
    # the instant enters only through f(t): at t and t + T the values agree
    assert np.max(np.abs(et(0.37, x) - et(0.37 + drv.period, x))) < 1e-9


def test_expect_tridiag_stationary_states():
    """Undriven (s = 0): the eigenvectors of the tridiagonal A = a0 H0 + a1 H1 (LAPACK's
    tridiagonal solver) give <v|A|v> = their eigenvalues exactly, at any t."""
    from scipy.linalg import eigh_tridiagonal
    nb = 40
    d, off, h1d = fi.dimer_matrices(nb, 1.0, U=0.05)
    a0, a1 = 1.3, 0.45
    lam, v = eigh_tridiagonal(a0 * d + a1 * h1d, a0 * off)
    ev = o.expect_tridiag(d, off, h1d, a0, a1, 0.0, fi.Drive(0.2, 1.1, 3.0))
    assert np.max(np.abs(ev(0.8, v.astype(np.complex128)) - lam)) < 1e-11 * np.max(np.abs(lam))


def test_adjoint1024_golden_plan_and_format():
    """The stored oracle gradient of the N = 1024 gate-fidelity workload (written once by
    tests/golden/make_golden.py adjoint1024, several CPU minutes) belongs to that workload's
    frozen plan: L, R, beta and Delta E recomputed here (cheap) match the file, and it holds a
    finite loss in [0, 1] and 256 finite gradient entries."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    g = mg.read_adjoint("adjoint1024.txt")
    a = fi.config_adjoint()
    plan = o.plan_piecewise(a.h0, a.h1, a.period, a.f)
    assert plan.L == int(g["L"])
    for k in ("R", "beta", "delta_e"):
        assert abs(getattr(plan, k) - g[k]) <= 1e-12 * abs(g[k])
    assert 0.0 <= g["loss"] <= 1.0 and len(g["g"]) == 256 and np.all(np.isfinite(g["g"]))


@pytest.mark.parametrize("steps", [2, 7, 40])
def test_single_level_is_the_phase_of_the_period_average(steps):
    """A single level (N = 1): every H(t) commutes, so U_T = exp(-i (h0 + h1 f_dc) T) (the
    cosine part of the drive integrates to zero over a period).  The 4th-order scheme gets it
    exactly, not just to O(h^4): the step midpoints of a cosine over a whole period sum to zero,
    and so do the f'' corrections.  A dropped phase or a wrong sign of beta fails it."""
    drv = fi.Drive(0.3, 1.5, 3.0, 0.4)
    a, b = np.array([0.7]), np.array([-1.3])
    p = o.plan_for_drive_tridiag(a, np.zeros(0), b, drv, steps)
    U = o.build_ut_tridiag(a, np.zeros(0), b, p)
    exact = np.exp(-1j * (a[0] + b[0] * drv.f_dc) * (2 * math.pi / drv.omega))
    assert abs(U[0, 0] - exact) <= 1e-14

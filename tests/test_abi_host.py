"""C-ABI library on the CPU: it loads, exports every symbol include/floquet.h declares, and its
host planner (stage a1: Magnus scalars, bounds, R, L, Bessel weights) agrees with the oracle.
No compute call needs a GPU here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest
from scipy.special import jv

import floquet_inputs as fi
import oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1508_07621_gb300", "libfloquet.so")


@pytest.fixture(scope="module")
def fq():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    import paper_1508_07621_gb300 as fq
    return fq


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "floquet.h")).read()
    return sorted(set(re.findall(r"\b(floquet_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(fq):
    names = declared_symbols()
    assert len(names) >= 12
    lib = ctypes.CDLL(LIB)
    for name in names:
        assert hasattr(lib, name), name


def test_dimer_plan_matches_oracle(fq):
    d = fi.config_dimer()
    prob, keep = fq.make_problem(d.n, fq.FQ_TRIDIAG, d.h0_diag, d.h1_diag, d.drive.period, d.steps,
                                 h0_off=d.h0_off, f_ac=1.5, omega=3.0, precision=fq.FQ_FP32)
    info, a = fq.floquet_plan_inspect(prob)
    p = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    assert info.L == p.L == 39
    assert abs(info.R - p.R) < 1e-12 * p.R
    assert abs(info.e_min - p.e_min) < 1e-9 * abs(p.e_min) and abs(info.e_max - p.e_max) < 1e-9 * p.e_max
    # Miller recurrence in the library vs the library routine J_l (scipy)
    ref = 2 * jv(np.arange(info.L + 1), info.R)
    ref[0] /= 2
    assert np.max(np.abs(a - ref)) < 1e-14


@pytest.mark.parametrize("R", [0.0, 1e-6, 0.0859, 2.5, 13.947, 60.0])
def test_library_bessel_and_order(fq, R):
    """Library L and a_l against scipy J_l for a problem whose R is set through user bounds."""
    n = 3
    h = 1.0
    prob, keep = fq.make_problem(n, fq.FQ_TRIDIAG, np.zeros(n), np.zeros(n), h, 1, h0_off=np.zeros(n - 1),
                                 f_ac=0.0, omega=1.0, e_min=-R if R > 0 else -1e-300, e_max=R if R > 0 else 1e-300)
    info, a = fq.floquet_plan_inspect(prob)
    assert info.L == o.chebyshev_order(info.R)
    ref = o.bessel_coefficients(info.R, info.L)
    assert np.max(np.abs(a - ref)) < 1e-14 * max(1.0, info.L)


def test_dense_plan_bounds_contain_exact(fq):
    """Lanczos bounds of the library contain the oracle's exact bounds and are tight (<1e-3)."""
    m = fi.config_goe64()
    prob, keep = fq.make_problem(64, fq.FQ_DENSE, m.h0, m.h1, m.drive.period, m.steps, f_ac=1.0, omega=1.0)
    info, _ = fq.floquet_plan_inspect(prob)
    p = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    assert info.e_min <= p.e_min and info.e_max >= p.e_max
    assert (info.e_max - info.e_min) < (p.e_max - p.e_min) * (1 + 1e-3)
    assert info.L == p.L


def test_argument_errors(fq):
    prob, keep = fq.make_problem(0, fq.FQ_DENSE, np.zeros(1), np.zeros(1), 1.0, 1)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_inspect(prob)
    assert e.value.status == fq.FQ_EINVAL
    prob, keep = fq.make_problem(4, fq.FQ_TRIDIAG, np.zeros(4), np.zeros(4), 1.0, 2, h0_off=np.zeros(3),
                                 precision=fq.FQ_BF16X3)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_inspect(prob)
    assert e.value.status == fq.FQ_EUNSUPPORTED
    for prec in (fq.FQ_BF16X6,):
        prob, keep = fq.make_problem(4, fq.FQ_TRIDIAG, np.zeros(4), np.zeros(4), 1.0, 2, h0_off=np.zeros(3),
                                     precision=prec)
        with pytest.raises(fq.FloquetError) as e:
            fq.floquet_plan_inspect(prob)
        assert e.value.status == fq.FQ_EUNSUPPORTED
    prob, keep = fq.make_problem(4, fq.FQ_DENSE, np.eye(4), np.eye(4), 1.0, 2, precision=fq.FQ_OZAKI + 1)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_inspect(prob)
    assert e.value.status == fq.FQ_EINVAL
    prob, keep = fq.make_problem(4, fq.FQ_DENSE, np.eye(4), np.eye(4), 1.0, 2, precision=fq.FQ_OZAKI)
    info, _ = fq.floquet_plan_inspect(prob)
    assert info.precision == fq.FQ_OZAKI


def test_fixed_chebyshev_terms(fq):
    """cheb_terms fixes L (the paper's timing runs use L = 50): the library's weights are then
    a_0 = J_0(R), a_l = 2 J_l(R) for l = 1..50 (scipy's Bessel functions), a value below the
    minimum L > R is raised to it, and out-of-range values are rejected."""
    from scipy.special import jv
    m = fi.config_goe_paper(64, 100)
    prob, keep = fq.make_problem(64, fq.FQ_DENSE, m.h0, m.h1, m.drive.period, m.steps, f_ac=1.0,
                                 omega=m.drive.omega, cheb_terms=50)
    info, a = fq.floquet_plan_inspect(prob)
    assert info.L == 50
    ref = np.array([jv(0, info.R)] + [2 * jv(l, info.R) for l in range(1, 51)])
    big = np.abs(ref) > 1e-290
    assert np.max(np.abs(a[big] - ref[big]) / np.abs(ref[big])) <= 1e-12
    prob, keep = fq.make_problem(64, fq.FQ_DENSE, m.h0, m.h1, m.drive.period, m.steps, f_ac=1.0,
                                 omega=m.drive.omega, cheb_terms=1)
    info, _ = fq.floquet_plan_inspect(prob)
    assert info.L == int(math.floor(info.R)) + 1
    for bad in (-1, 1025):
        prob, keep = fq.make_problem(64, fq.FQ_DENSE, m.h0, m.h1, 2.0, 10, cheb_terms=bad)
        with pytest.raises(fq.FloquetError) as e:
            fq.floquet_plan_inspect(prob)
        assert e.value.status == fq.FQ_EINVAL


@pytest.mark.parametrize("case,status", [
    ("steps0", "FQ_EINVAL"), ("period0", "FQ_EINVAL"), ("format9", "FQ_EINVAL"), ("drive9", "FQ_EINVAL"),
    ("piecewise_without_f", "FQ_EINVAL"), ("order5", "FQ_EINVAL"), ("order6_tridiag_fp32", "FQ_EUNSUPPORTED"),
    ("order6_piecewise", "FQ_EUNSUPPORTED"), ("tile96", "FQ_EINVAL"), ("tilek48", "FQ_EINVAL"),
    ("dense_fp32", "FQ_EUNSUPPORTED"),
    ("tridiag_x6", "FQ_EUNSUPPORTED"), ("kernel9", "FQ_EINVAL")])
def test_problem_validation(fq, case, status):
    """Every rejected problem fails in host planning with its status and a message, before any
    device work."""
    n = 8
    d = np.arange(n, dtype=float)
    g = fi.goe(n, 5)
    kw = dict(f_ac=1.0, omega=1.0)
    if case == "steps0":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 0, **kw)
    elif case == "period0":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 0.0, 4, **kw)
    elif case == "format9":
        prob, keep = fq.make_problem(n, 9, g, g, 1.0, 4, **kw)
    elif case == "drive9":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, drive_kind=9, **kw)
    elif case == "piecewise_without_f":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, drive_kind=fq.FQ_DRIVE_PIECEWISE, **kw)
    elif case == "order5":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, magnus_order=5, **kw)
    elif case == "order6_tridiag_fp32":
        prob, keep = fq.make_problem(n, fq.FQ_TRIDIAG, d, d, 1.0, 4, h0_off=np.ones(n - 1), magnus_order=6,
                                     precision=fq.FQ_FP32, **kw)
    elif case == "order6_piecewise":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, drive_kind=fq.FQ_DRIVE_PIECEWISE,
                                     f_steps=np.ones(4), magnus_order=6)
    elif case == "tile96":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, precision=fq.FQ_BF16X3, tile_n=96, **kw)
    elif case == "tilek48":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, precision=fq.FQ_BF16X3, tile_k=48, **kw)
    elif case == "dense_fp32":
        prob, keep = fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, precision=fq.FQ_FP32, **kw)
    elif case == "kernel9":
        prob, keep = fq.make_problem(n, fq.FQ_TRIDIAG, d, d, 1.0, 4, h0_off=np.ones(n - 1), kernel=9, **kw)
    else:
        prob, keep = fq.make_problem(n, fq.FQ_TRIDIAG, d, d, 1.0, 4, h0_off=np.ones(n - 1),
                                     precision=fq.FQ_BF16X6, **kw)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_inspect(prob)
    assert e.value.status == getattr(fq, status)
    assert fq.floquet_last_error()


NAN, INF = float("nan"), float("inf")


@pytest.mark.parametrize("case,status", [
    ("f_ac_nan", "FQ_EINVAL"), ("omega_inf", "FQ_EINVAL"), ("phi0_nan", "FQ_EINVAL"), ("period_inf", "FQ_EINVAL"),
    ("h0_nan_dense", "FQ_EINVAL"), ("h1_inf_dense", "FQ_EINVAL"), ("h0_nan_tridiag", "FQ_EINVAL"),
    ("h0_off_inf", "FQ_EINVAL"), ("f_steps_nan", "FQ_EINVAL"), ("user_bounds_inf", "FQ_EINVAL"),
    ("overflowing_bounds", "FQ_EUNSUPPORTED"), ("R_above_cap", "FQ_EUNSUPPORTED")])
def test_non_finite_and_oversized_problems(fq, case, status):
    """A NaN or Inf anywhere in the problem, bounds that overflow, or an R = h Delta E beyond what
    any step can hold (about R + 300 products) are rejected in host planning with a message;
    none of them may hang the search for L or abort the process."""
    n = 8
    g = fi.goe(n, 5)
    d = np.arange(n, dtype=float)
    off = np.ones(n - 1)
    kw = dict(f_ac=1.0, omega=1.0)
    bad = lambda a, v: np.where(np.arange(a.size).reshape(a.shape) == a.size // 2, v, a)
    make = {
        "f_ac_nan": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, f_ac=NAN, omega=1.0),
        "omega_inf": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, f_ac=1.0, omega=INF),
        "phi0_nan": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, phi0=NAN, **kw),
        "period_inf": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, INF, 4, **kw),
        "h0_nan_dense": lambda: fq.make_problem(n, fq.FQ_DENSE, bad(g, NAN), g, 1.0, 4, **kw),
        "h1_inf_dense": lambda: fq.make_problem(n, fq.FQ_DENSE, g, bad(g, INF), 1.0, 4, **kw),
        "h0_nan_tridiag": lambda: fq.make_problem(n, fq.FQ_TRIDIAG, bad(d, NAN), d, 1.0, 4, h0_off=off, **kw),
        "h0_off_inf": lambda: fq.make_problem(n, fq.FQ_TRIDIAG, d, d, 1.0, 4, h0_off=bad(off, INF), **kw),
        "f_steps_nan": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, drive_kind=fq.FQ_DRIVE_PIECEWISE,
                                               f_steps=np.array([1.0, NAN, 1.0, 1.0])),
        "user_bounds_inf": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, e_min=-1.0, e_max=INF, **kw),
        "overflowing_bounds": lambda: fq.make_problem(n, fq.FQ_DENSE, g, g, 1.0, 4, e_min=-1.7e308, e_max=1.7e308,
                                                      **kw),
        "R_above_cap": lambda: fq.make_problem(n, fq.FQ_DENSE, g * 1e6, g, 1.0, 1, **kw),
    }
    prob, keep = make[case]()
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_inspect(prob)
    assert e.value.status == getattr(fq, status)
    assert fq.floquet_last_error()


def test_largest_accepted_R(fq):
    """Just below the cap the plan is accepted, with L = the smallest l > R whose next Bessel
    weight is below the tolerance (scipy's J_l as the check)."""
    from scipy.special import jv
    prob, keep = fq.make_problem(2, fq.FQ_DENSE, np.eye(2), np.zeros((2, 2)), 1.0, 1, f_ac=1.0, omega=1.0,
                                 e_min=-16000.0, e_max=16000.0)
    info, a = fq.floquet_plan_inspect(prob, cap=20000)
    assert info.R == pytest.approx(16000.0) and info.L > 16000
    assert abs(jv(info.L + 1, info.R)) < 1e-14 and abs(jv(info.L, info.R)) >= 1e-14


def test_plan_create_rejects_before_device_work(fq):
    """An invalid problem fails in floquet_plan_create's host planning with the same status as in
    floquet_plan_inspect, without needing a device, and leaves no plan behind."""
    g = fi.goe(4, 5)
    prob, keep = fq.make_problem(4, fq.FQ_DENSE, g, g, 1.0, 4, f_ac=NAN, omega=1.0)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_create(prob)
    assert e.value.status == fq.FQ_EINVAL and "finite" in fq.floquet_last_error()


def _built_spectrum(n, seed, theta):
    """U = V diag(e^{-i theta}) V^H with Haar V: quasienergies theta/T and states V known by
    construction (Eq. 5)."""
    v = fi.haar_unitary(n, seed)
    return (v * np.exp(-1j * theta)[None, :]) @ v.conj().T, v


@pytest.mark.parametrize("n", [1, 2, 7, 64, 200])
def test_host_quasienergies_known_spectrum(fq, n):
    """The library's host Schur solver recovers a spectrum fixed by construction (eps = theta/T,
    ascending in [-pi/T, pi/T)), with orthonormal states that satisfy U phi = e^{-i eps T} phi
    and match the constructed eigenvectors up to phase; eps alone gives the same values."""
    T = 2.5
    theta = np.sort(np.random.default_rng(n).uniform(-math.pi, math.pi, n))
    u, v = _built_spectrum(n, 40 + n, theta)
    eps, st = fq.floquet_quasienergies(u, T)
    assert np.all(np.diff(eps) >= 0)
    assert np.max(np.abs(eps - theta / T)) <= 1e-12
    assert np.max(np.abs(u @ st.T - st.T * np.exp(-1j * eps * T)[None, :])) <= 1e-12
    assert np.max(np.abs(st.conj() @ st.T - np.eye(n))) <= 1e-12
    gap = np.min(np.diff(np.concatenate([theta, [theta[0] + 2 * math.pi]]))) if n > 1 else 1.0
    if gap > 1e-6:  # well separated: each state is the constructed column up to a phase
        assert np.max(np.abs(np.abs(np.sum(st.conj() * v.T, axis=1)) - 1)) <= 1e-12 / gap
    eps2, none = fq.floquet_quasienergies(u, T, states=False)
    assert none is None and np.max(np.abs(eps2 - eps)) <= 1e-12


def test_host_quasienergies_special_cases(fq):
    """Closed forms: the cyclic shift has the N-th roots of unity as eigenvalues; the identity
    is fully degenerate (eps = 0, any orthonormal basis); a diagonal U is already in Schur form,
    including the branch point theta = -pi (lambda = -1 maps to eps = -pi/T, not +pi/T)."""
    n = 12
    shift = np.roll(np.eye(n), 1, axis=0).astype(complex)
    eps, st = fq.floquet_quasienergies(shift, 1.0)
    ref = np.sort(np.array([-(2 * math.pi * k / n) for k in range(n)]))
    ref = np.sort(np.where(ref < -math.pi, ref + 2 * math.pi, ref))
    assert np.max(np.abs(eps - ref)) <= 1e-13
    eps, st = fq.floquet_quasienergies(np.eye(5, dtype=complex), 3.0)
    assert np.max(np.abs(eps)) == 0 and np.max(np.abs(st.conj() @ st.T - np.eye(5))) <= 1e-15
    d = np.exp(-1j * np.array([0.5, -math.pi, 2.0]))
    d[1] = -1.0
    eps, st = fq.floquet_quasienergies(np.diag(d), 2.0)
    assert np.allclose(eps, np.array([-math.pi, 0.5, 2.0]) / 2.0, atol=1e-15, rtol=0)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_quasienergies(np.eye(3, dtype=complex), 0.0)
    assert e.value.status == fq.FQ_EINVAL


def test_host_quasienergies_of_oracle_UT(fq):
    """On a propagated U_T (GOE64 drive, the oracle's FP64 chain), the library's quasienergies
    equal the oracle's (LAPACK zgeev)."""
    m = fi.config_goe64()
    p = o.plan_for_drive_dense(m.h0, m.h1, m.drive, 40)
    u = o.build_ut_dense(m.h0, m.h1, p)
    T = m.drive.period
    eps, _ = fq.floquet_quasienergies(u, T, states=False)
    assert np.max(np.abs(eps - o.quasienergies(u, T))) <= 1e-12


def test_binding_refuses_bad_buffers(fq):
    """The binding hands raw pointers to the library, so it refuses, with FQ_EINVAL and before any
    call into it, a host tensor where device memory is expected, host arrays shorter than the
    problem implies, and a non-square U_T for the host eigensolver."""
    import torch
    d = np.arange(6, dtype=float)
    prob, keep = fq.make_problem(6, fq.FQ_TRIDIAG, d, d, 1.0, 4, h0_off=np.ones(5), f_ac=1.0, omega=1.0,
                                 precision=fq.FQ_FP32)
    host_u = torch.zeros((6, 6), dtype=torch.complex128)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_build_UT_static(prob, host_u)
    assert e.value.status == fq.FQ_EINVAL and "CUDA tensor" in str(e.value)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_unitarity_defect(host_u, 6, None, 6, torch.zeros(256, dtype=torch.uint8))
    assert e.value.status == fq.FQ_EINVAL and "CUDA tensor" in str(e.value)
    g = fi.goe(8, 5)
    for kw in (dict(h0=g[:7]), dict(h1=g.ravel()[:63]), dict(h0_off=np.ones(6), fmt=fq.FQ_TRIDIAG),
               dict(f_steps=np.ones(3), drive_kind=fq.FQ_DRIVE_PIECEWISE)):
        fmt = kw.pop("fmt", fq.FQ_DENSE)
        args = dict(h0=np.diag(g) if fmt == fq.FQ_TRIDIAG else g, h1=np.diag(g) if fmt == fq.FQ_TRIDIAG else g)
        args.update({k: v for k, v in kw.items() if k in ("h0", "h1")})
        extra = {k: v for k, v in kw.items() if k not in ("h0", "h1")}
        with pytest.raises(ValueError):
            fq.make_problem(8, fmt, args["h0"], args["h1"], 1.0, 4, **extra)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_quasienergies(np.eye(3, 4, dtype=complex), 1.0)
    assert e.value.status == fq.FQ_EINVAL


def test_host_quasienergies_concurrent_calls(fq):
    """Calls from several host threads at once (ctypes releases the GIL) each get their own
    worker pool and return exactly what a lone call returns."""
    import concurrent.futures as cf
    us = [fi.haar_unitary(160, 900 + i) for i in range(4)]
    alone = [fq.floquet_quasienergies(u, 1.0) for u in us]
    with cf.ThreadPoolExecutor(4) as ex:
        together = list(ex.map(lambda u: fq.floquet_quasienergies(u, 1.0), us))
    for (e1, s1), (e2, s2) in zip(alone, together):
        assert np.array_equal(e1, e2) and np.array_equal(s1, s2)


def test_library_bessel_sweep_to_the_R_cap(fq):
    """Across R = 1e-8 .. 16000 (up to the planning cap): the library's L equals the oracle's
    truncation rule (smallest l > R with |J_{l+1}(R)| < 1e-14), and every weight a_l equals
    scipy's (2 -) J_l(R) to 16 eps sqrt(L) absolute: Miller's recurrence is stable downward for
    any R, and its rounding (like scipy's) accumulates as a random walk over the ~L steps (about
    9 eps sqrt(L) seen at R = 16000)."""
    from scipy.special import jv
    n, h = 2, 1.0
    for R in np.concatenate([np.logspace(-8, 4, 25), [12345.6, 16000.0]]):
        prob, keep = fq.make_problem(n, fq.FQ_TRIDIAG, np.zeros(n), np.zeros(n), h, 1, h0_off=np.zeros(n - 1),
                                     f_ac=0.0, omega=1.0, e_min=-R, e_max=R)
        info, a = fq.floquet_plan_inspect(prob, cap=20000)
        assert abs(info.R - R) <= 1e-15 * R
        assert info.L == o.chebyshev_order(info.R), R
        ref = jv(np.arange(info.L + 1), info.R)
        ref[1:] *= 2
        assert np.max(np.abs(a - ref)) <= 16 * 2.2e-16 * math.sqrt(info.L) + 1e-18, (R, np.max(np.abs(a - ref)))


def test_tridiag_order6_bounds_contain_the_exact_ones(fq):
    """A tridiagonal plan of the 6th-order scheme: the host's bounds of Omega_m / h (Sturm bounds
    of H0 + g H1 widened by every commutator band's largest row sum) contain the exact extreme
    eigenvalues over all steps (the oracle's dense Omega_m through LAPACK), and L is at least the
    oracle's."""
    d = fi.config_dimer(nb=30, steps=40)
    drv = fi.Drive(0.2, 1.5, 3.0, 0.4)
    prob, keep = fq.make_problem(d.n, fq.FQ_TRIDIAG, d.h0_diag, d.h1_diag, drv.period, d.steps, h0_off=d.h0_off,
                                 f_dc=drv.f_dc, f_ac=drv.f_ac, omega=drv.omega, phi0=drv.phi0, magnus_order=6)
    info, _ = fq.floquet_plan_inspect(prob)
    h0 = np.diag(d.h0_diag) + np.diag(d.h0_off, 1) + np.diag(d.h0_off, -1)
    rp, _ = o.plan_dense6(h0, np.diag(d.h1_diag), drv, d.steps)
    lo, hi = rp.beta - rp.delta_e, rp.beta + rp.delta_e
    assert info.e_min <= lo and info.e_max >= hi
    assert info.L >= rp.L

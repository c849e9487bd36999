"""Second propagation round: period averages <A>_T of Floquet states (Eq. 17) through the C ABI,
against the oracle on the same states, and the Floquet Hellmann-Feynman relation
d eps / d f_dc = <H1>_T measured entirely on the GPU path."""
import math

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


@pytest.mark.parametrize("precision", ["FQ_FP64", "FQ_DF32", "FQ_OZAKI"])
def test_dense_fp64_averages_match_oracle(fq, precision):
    """Period averages through the FP64 chain and the two emulated ones (same FP64 criterion)."""
    n, M = 40, 60
    h0, h1 = fi.goe(n, 1401), fi.goe(n, 1402)
    drv = fi.Drive(0.1, 1.1, 1.2, 0.3)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         precision=getattr(fq, precision))
    eps, states = fq.floquet_states(plan.build_UT(), drv.period)
    e_avg = plan.average_observable(states, 1.0, 0.0, 1.0).cpu().numpy()       # <H(t)>_T
    h1_avg = plan.average_observable(states, 0.0, 1.0, 0.0).cpu().numpy()      # <H1>_T
    p = o.plan_for_drive_dense(h0, h1, drv, M)
    k = o.commutator_dense(h0, h1)
    step = lambda m, x: o.chebyshev_step(lambda v: o.omega_tilde_dense(h0, h1, k, p, m) @ v, x, p.coeffs, p.phase)
    x0 = states.cpu().numpy().T
    ref_e = o.average_observable(step, o.expect_dense(h0, h1, 1.0, 0.0, 1.0, drv), x0, drv, M)
    ref_h1 = o.average_observable(step, o.expect_dense(h0, h1, 0.0, 1.0, 0.0, drv), x0, drv, M)
    assert np.max(np.abs(e_avg - ref_e)) <= 1e-10
    assert np.max(np.abs(h1_avg - ref_h1)) <= 1e-10


def test_hellmann_feynman_on_gpu(fq):
    """All on the library: U_T at f_dc +- d (FP64 dense), quasienergy slopes vs <H1>_T."""
    n, M = 24, 80
    h0, h1 = fi.goe(n, 1501), fi.goe(n, 1502)

    def run(fdc):
        plan = fq.Plan.dense(h0, h1, omega=1.3, f_ac=0.9, f_dc=fdc, steps=M)
        eps, st = fq.floquet_states(plan.build_UT(), 2 * math.pi / 1.3)
        return plan, eps, st

    fdc, d = 0.2, 1e-4
    plan, eps, states = run(fdc)
    _, ep, _ = run(fdc + d)
    _, em, _ = run(fdc - d)
    near = lambda e0, e1: np.array([e1[np.argmin(np.abs(np.angle(np.exp(1j * (e1 - x) * 2 * math.pi / 1.3))))]
                                    for x in e0])
    slope = (near(eps, ep) - near(eps, em)) / (2 * d)
    h1_avg = plan.average_observable(states, 0.0, 1.0, 0.0).cpu().numpy()
    assert np.max(np.abs(slope - h1_avg)) < 1e-6


@pytest.mark.parametrize("precision,kernel", [(0, 1), (1, 2)])
def test_dimer_average_energy(fq, precision, kernel):
    """Dimer (dim 41, M = 100): <H(t)>_T of its Floquet states (the paper's sorting key, §7), FP64
    streaming and FP32 resident, against the oracle.  A state error e moves <H> by at most
    2 ||H|| e, so the FP32 tolerance is 2 ||H|| min(1e-5, the FP32 rounding bound of the states)."""
    d = fi.config_dimer(nb=40, steps=100)
    plan = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=3.0, f_ac=1.5, steps=d.steps,
                           precision=precision, kernel=kernel)
    ref_plan = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=3.0, f_ac=1.5, steps=d.steps, precision=0,
                               kernel=1)
    eps, states = fq.floquet_states(ref_plan.build_UT(), d.drive.period)
    avg = plan.average_observable(states, 1.0, 0.0, 1.0).cpu().numpy()
    p = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    kl = o.commutator_tridiag(d.h0_off, d.h1_diag)

    def step(m, x):
        dd, lo = o.omega_tilde_tridiag(d.h0_diag, d.h0_off, d.h1_diag, kl, p, m)
        return o.chebyshev_step(lambda v: o.apply_tridiag(dd, lo, v), x, p.coeffs, p.phase)

    ref = o.average_observable(step, o.expect_tridiag(d.h0_diag, d.h0_off, d.h1_diag, 1.0, 0.0, 1.0, d.drive),
                               states.cpu().numpy().T, d.drive, d.steps)
    if precision == 0:
        tol = 1e-9
    else:
        hn = max(abs(plan.info.e_min), abs(plan.info.e_max))
        tol = 2 * hn * min(1e-5, 2 * d.steps * plan.info.R * U32 + 4 * math.sqrt(d.steps) * plan.info.L * U32)
    assert np.max(np.abs(avg - ref)) <= tol
    order = np.argsort(avg)      # the paper sorts Floquet states by mean energy
    assert len(set(order.tolist())) == d.n


def test_floquet_analysis_sorted_by_average_energy(fq):
    """floquet_analysis: U_T, Floquet states, <H(t)>_T by the second round, sorted ascending;
    energies match the oracle's averages of the same states and the order is by energy."""
    n, M = 32, 50
    h0, h1 = fi.goe(n, 1801), fi.goe(n, 1802)
    drv = fi.Drive(0.3, 1.0, 1.4, 0.2)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M)
    avg, eps, states = fq.floquet_analysis(plan)
    assert np.all(np.diff(avg) >= 0)
    p = o.plan_for_drive_dense(h0, h1, drv, M)
    k = o.commutator_dense(h0, h1)
    step = lambda m, x: o.chebyshev_step(lambda v: o.omega_tilde_dense(h0, h1, k, p, m) @ v, x, p.coeffs, p.phase)
    ref = o.average_observable(step, o.expect_dense(h0, h1, 1.0, 0.0, 1.0, drv), states.cpu().numpy().T, drv, M)
    assert np.max(np.abs(avg - ref)) <= 1e-10
    # each row is a Floquet state: U_T phi = e^{-i eps T} phi
    U = plan.build_UT().cpu().numpy()
    phi = states.cpu().numpy()
    res = U @ phi.T - phi.T * np.exp(-1j * eps * drv.period)[None, :]
    assert np.max(np.abs(res)) < 1e-9


@pytest.mark.parametrize("precision", [0, 2])
def test_overlap_phase_error_matches_oracle(fq, precision):
    """Eq. 20 on the library (coarse chain applied to the fine Floquet states by
    floquet_propagate) against the oracle's Sigma from its own U_T's.  FP64 to 1e-9; the BF16X3
    coarse chain to sqrt(N) 1e-5: the split target bounds U_T's entries by 1e-5, hence
    ||dU phi||_2 <= sqrt(N) 1e-5 for a unit phi, and |dSigma| <= ||dU phi||_2."""
    n, M = 24, 40
    h0, h1 = fi.goe(n, 1901), fi.goe(n, 1902)
    drv = fi.Drive(0.2, 1.2, 1.3, 0.4)
    coarse = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                           precision=precision)
    fine = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=2 * M)
    eps, sig = fq.overlap_phase_error(coarse, fine.build_UT())
    uc = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M))
    uf = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, 2 * M))
    ref_eps, ref_sig = o.overlap_phase_error(uc, uf, drv.period)
    assert np.max(np.abs(eps - ref_eps)) < 1e-10
    assert np.max(np.abs(sig - ref_sig)) <= (1e-9 if precision == 0 else math.sqrt(n) * 1e-5)
    assert np.max(ref_sig) > 1e-7   # the test resolves the coarse chain's error

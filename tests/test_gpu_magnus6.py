"""The paper's own 6th-order scheme (Eq. 14 in full, reading R12: alphas as Gauss-Legendre
moments) on the GPU: FP64 parity with the oracle's order-6 chain, observed order 6 against an
independent RK4 solution, and the BF16X6 tensor-core path with the same scheme; for dense plans
and for tridiagonal ones (the dimer the paper runs with this scheme)."""
import math
import sys
import os

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_pins import rk4_propagator  # noqa: E402  (textbook integrator, tests only)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


def test_magnus6_fp64_matches_oracle(fq):
    n, M = 12, 16
    h0, h1 = fi.goe(n, 1601), fi.goe(n, 1602)
    drv = fi.Drive(0.2, 1.4, 1.1, 0.5)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         magnus_order=6)
    U = plan.build_UT().cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    rp, oms = o.plan_dense6(h0, h1, drv, M)
    assert np.max(np.abs(U - o.build_ut_dense6(rp, oms))) <= 1e-10


def test_magnus6_order_on_gpu(fq):
    h0, h1 = fi.goe(4, 11), fi.goe(4, 12)
    drv = fi.Drive(0.3, 1.2, 1.3, 0.7)
    ref = rk4_propagator(h0, h1, drv, drv.period, 1 << 15)
    errs = []
    for M in (8, 16, 32):
        plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                             magnus_order=6)
        errs.append(np.max(np.abs(plan.build_UT().cpu().numpy() - ref)))
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 50.0 < r < 80.0, errs


def test_magnus6_split_bf16x6(fq):
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=m.steps, precision=fq.FQ_BF16X6, magnus_order=6)
    U = plan.build_UT().cpu().numpy()
    rp, oms = o.plan_dense6(m.h0, m.h1, m.drive, m.steps)
    ref = o.build_ut_dense6(rp, oms)
    eps = 2.0 ** -23
    tol = min(1e-5, 2 * m.steps * plan.info.R * eps + 4 * math.sqrt(m.steps * plan.info.L) * eps)  # split target
    assert np.max(np.abs(U - ref)) <= tol


def _dense(d):
    return np.diag(d.h0_diag) + np.diag(d.h0_off, 1) + np.diag(d.h0_off, -1), np.diag(d.h1_diag)


def _tri6(fq, d, drv, **kw):
    return fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc,
                           phi0=drv.phi0, steps=d.steps, magnus_order=6, **kw)


def test_magnus6_tridiagonal_matches_oracle(fq):
    """A tridiagonal plan of the 6th-order scheme (heptadiagonal Omega~ from banded commutators,
    streaming FP64 kernel): the whole dim-41 U_T against the oracle's order-6 chain on the same
    matrices in dense form, at the FP64 criterion."""
    d = fi.config_dimer(nb=40, steps=60)
    drv = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = _tri6(fq, d, drv)
    U = plan.build_UT().cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    rp, oms = o.plan_dense6(*_dense(d), drv, d.steps)
    err = np.max(np.abs(U - o.build_ut_dense6(rp, oms)))
    print(f"order-6 tridiagonal dim 41: max err {err:.2e}, L = {plan.info.L} (oracle {rp.L})")
    assert err <= 1e-10


def test_magnus6_tridiagonal_sampled_columns(fq):
    """dim 301 (bands of half-width 3 across several 256-row kernel blocks), M = 100: three columns
    of U_T against the oracle's order-6 chain."""
    d = fi.config_dimer(nb=300, steps=100)
    drv = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = _tri6(fq, d, drv)
    U = plan.build_UT().cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    cols = [0, 150, 300]
    h0, h1 = _dense(d)
    rp, oms = o.plan_dense6(h0, h1, drv, d.steps)
    x = np.eye(d.n, dtype=complex)[:, cols]
    for om in oms:  # the oracle's build_ut_dense6 on three columns
        omt = (om / rp.h - rp.beta * np.eye(d.n)) / rp.delta_e
        x = o.chebyshev_step(lambda v: omt @ v, x, rp.coeffs, rp.phase)
    err = np.max(np.abs(U[:, cols] - x))
    print(f"order-6 tridiagonal dim 301: max err {err:.2e}")
    assert err <= 1e-10


def test_magnus6_tridiagonal_order_on_gpu(fq):
    """Observed order 6 of the tridiagonal path: the error against an RK4 solution falls by about
    2^6 per halving of h (M = 16, 32, 64 on the dim-9 dimer)."""
    d = fi.config_dimer(nb=8, steps=16)
    drv = fi.Drive(0.3, 1.2, 1.3, 0.7)
    ref = rk4_propagator(*_dense(d), drv, drv.period, 1 << 15)
    errs = []
    for M in (16, 32, 64):
        d.steps = M
        plan = _tri6(fq, d, drv)
        errs.append(np.max(np.abs(plan.build_UT().cpu().numpy() - ref)))
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 50.0 < r < 80.0, errs


def test_magnus6_tridiagonal_needs_fp64_streaming(fq):
    """6th-order tridiagonal plans run in FQ_FP64 on the streaming kernel only."""
    d = fi.config_dimer(nb=20, steps=10)
    drv = fi.Drive(0.2, 1.5, 3.0, 0.4)
    for kw in (dict(precision=fq.FQ_FP32), dict(precision=fq.FQ_OZAKI), dict(precision=fq.FQ_DF32),
               dict(kernel=fq.FQ_KERNEL_RESIDENT), dict(kernel=fq.FQ_KERNEL_TILED), dict(kernel=fq.FQ_KERNEL_BAND)):
        with pytest.raises(fq.FloquetError) as e:
            _tri6(fq, d, drv, **kw)
        assert e.value.status == fq.FQ_EUNSUPPORTED, kw

"""The paper's own 6th-order scheme (Eq. 14 in full, reading R12: alphas as Gauss-Legendre
moments) on the GPU: FP64 parity with the oracle's order-6 chain, observed order 6 against an
independent RK4 solution, and the BF16X6 tensor-core path with the same scheme."""
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


def test_magnus6_rejects_tridiagonal(fq):
    d = fi.config_dimer(nb=20, steps=10)
    prob, keep = fq.make_problem(d.n, fq.FQ_TRIDIAG, d.h0_diag, d.h1_diag, d.drive.period, d.steps, h0_off=d.h0_off,
                                 f_ac=1.5, omega=3.0, precision=fq.FQ_FP32, magnus_order=6)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_inspect(prob)
    assert e.value.status == fq.FQ_EUNSUPPORTED

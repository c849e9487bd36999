"""Degenerate sizes of the tridiagonal chain on the GPU: a single level (N = 1, where U_T is the
phase exp(-i (h0 + h1 f_dc) T) exactly, since the step midpoints, and the Gauss nodes of the
6th-order scheme, of a cosine over a whole period sum to zero) on every tridiagonal kernel; one
state; an empty block of states."""
import math

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1508_07621_gb300 as fq
    return fq


DRV = fi.Drive(0.3, 1.5, 3.0, 0.4)


@pytest.mark.parametrize("precision,kernel,order,tol", [
    ("FQ_OZAKI", "FQ_KERNEL_AUTO", 0, 1e-12),      # band kernel
    ("FQ_FP64", "FQ_KERNEL_AUTO", 0, 1e-12),       # tiled FP64
    ("FQ_FP64", "FQ_KERNEL_STREAM", 0, 1e-12),     # streaming FP64
    ("FQ_DF32", "FQ_KERNEL_AUTO", 0, 1e-12),       # double-float tiled
    ("FQ_FP32", "FQ_KERNEL_AUTO", 0, 1e-6),        # resident FP32
    ("FQ_FP64", "FQ_KERNEL_AUTO", 6, 1e-12),       # 6th order, heptadiagonal streaming FP64
])
def test_single_level_is_the_period_phase(fq, precision, kernel, order, tol):
    a, b = np.array([0.7]), np.array([-1.3])
    plan = fq.Plan.tridiag(a, np.zeros(0), b, omega=DRV.omega, f_ac=DRV.f_ac, f_dc=DRV.f_dc, phi0=DRV.phi0,
                           steps=40, precision=getattr(fq, precision), kernel=getattr(fq, kernel),
                           magnus_order=order)
    U = plan.build_UT().cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    exact = np.exp(-1j * (a[0] + b[0] * DRV.f_dc) * (2 * math.pi / DRV.omega))
    assert U.shape == (1, 1) and abs(U[0, 0] - exact) <= tol


def test_band_one_state_and_an_empty_block(fq):
    """The band path with a single state (dim 701, 3 steps) against the oracle, and with no
    states at all (a call that does nothing and leaves its output untouched)."""
    import torch
    d = fi.config_dimer(nb=700, steps=200)
    d.drive = DRV
    plan = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=DRV.omega, f_ac=DRV.f_ac, f_dc=DRV.f_dc,
                           phi0=DRV.phi0, steps=d.steps, precision=fq.FQ_OZAKI)
    n = d.n
    x0 = np.exp(2j * np.pi * fi.uniform(2901, n)) / np.sqrt(n)
    X0 = torch.from_numpy(x0[None, :].astype(np.complex128)).cuda()
    X = plan.propagate(X0, 0, 3).cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, DRV, d.steps)
    ref = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x0[:, None], 0, 3)[:, 0]
    assert np.max(np.abs(X[0] - ref)) <= 1e-10
    ws = fq.workspace(plan.workspace_size(1))
    out = torch.full((1, n), 7.0, dtype=torch.complex128, device="cuda")
    fq.floquet_propagate(plan.handle, X0, out, 0, 0, 3, ws)
    torch.cuda.synchronize()
    assert plan.check_status() == fq.FQ_OK
    assert bool((out == 7.0).all())

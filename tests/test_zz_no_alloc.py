"""floquet_build_UT_static: the entry point for callers that cannot call cudaMalloc.

It keeps all of its scratch in the library's static device array instead of a caller
workspace.  Checked here against floquet_build_UT (plan + workspace) on the same problem,
through the C ABI, on two calls in a row with different problems (the array keeps the previous
call's contents, so the second call must not see them), and for the size limit.
This file is collected last so that a failure here does not stop the other GPU tests.
"""
import math

import numpy as np
import pytest

import floquet_inputs as fi

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def tol_f32(M, L, R):
    """min(1e-5, 2 M R u + 4 sqrt(M) L u): the FP32 rounding bound, capped at the FP32-level target."""
    return min(1e-5, 2.0 * M * R * U32 + 4.0 * math.sqrt(M) * L * U32)


def _problem(fq, d):
    return fq.make_problem(d.n, fq.FQ_TRIDIAG, d.h0_diag, d.h1_diag, d.drive.period, d.steps, h0_off=d.h0_off,
                           f_dc=d.drive.f_dc, f_ac=d.drive.f_ac, omega=d.drive.omega, phi0=d.drive.phi0,
                           precision=fq.FQ_FP32, kernel=fq.FQ_KERNEL_RESIDENT)


def test_static_entry_matches_workspace_entry():
    import torch
    import paper_1508_07621_gb300 as fq
    assert torch.cuda.is_available()
    cases = [fi.config_dimer(nb=700, steps=300), fi.config_dimer(nb=40, steps=100)]
    cases[1].drive = fi.Drive(0.3, 1.5, 3.0, 0.5)
    for d in cases:
        prob, keep = _problem(fq, d)
        plan = fq.Plan(prob, keep)
        ref = plan.build_UT()
        U = torch.full((d.n, d.n), float("nan"), dtype=torch.complex128, device="cuda")
        fq.floquet_build_UT_static(prob, U)
        err = (U - ref).abs().max().item()
        assert err <= tol_f32(d.steps, plan.info.L, plan.info.R), err
        plan.close()


def test_static_entry_rejects_oversize():
    import torch
    import paper_1508_07621_gb300 as fq
    d = fi.config_dimer(nb=10000, steps=2000)     # (2 * 2000 + 1) * 10240 padded rows * 8 B = 328 MB > 16 MiB
    prob, keep = _problem(fq, d)
    U = torch.empty((d.n, d.n), dtype=torch.complex128, device="cuda")
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_build_UT_static(prob, U)
    assert e.value.status == fq.FQ_EINVAL and "floquet_build_UT_static" in fq.floquet_last_error()


def test_static_entry_rejects_other_kernels():
    """The entry point runs the resident kernel only: a problem asking for another one is refused."""
    import torch
    import paper_1508_07621_gb300 as fq
    d = fi.config_dimer(nb=40, steps=100)
    U = torch.empty((d.n, d.n), dtype=torch.complex128, device="cuda")
    for kernel in (fq.FQ_KERNEL_STREAM, fq.FQ_KERNEL_TILED):
        prob, keep = fq.make_problem(d.n, fq.FQ_TRIDIAG, d.h0_diag, d.h1_diag, d.drive.period, d.steps,
                                     h0_off=d.h0_off, f_ac=d.drive.f_ac, omega=d.drive.omega,
                                     precision=fq.FQ_FP32, kernel=kernel)
        with pytest.raises(fq.FloquetError) as e:
            fq.floquet_build_UT_static(prob, U)
        assert e.value.status == fq.FQ_EUNSUPPORTED


def test_static_entry_allocates_no_device_memory():
    """The property the entry point exists for: after a first call on the device (which looks up
    the array), another call on a different problem leaves the device's free memory unchanged."""
    import torch
    import paper_1508_07621_gb300 as fq
    a, b = fi.config_dimer(nb=300, steps=200), fi.config_dimer(nb=500, steps=150)
    Ua = torch.empty((a.n, a.n), dtype=torch.complex128, device="cuda")
    Ub = torch.empty((b.n, b.n), dtype=torch.complex128, device="cuda")
    pa, keep_a = _problem(fq, a)
    pb, keep_b = _problem(fq, b)
    fq.floquet_build_UT_static(pa, Ua)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fq.floquet_build_UT_static(pb, Ub)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.isfinite(torch.view_as_real(Ub)).all()

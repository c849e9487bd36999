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
    return 2.0 * M * R * U32 + 4.0 * math.sqrt(M) * L * U32


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
    d = fi.config_dimer(nb=10000, steps=2000)     # 3 * 2000 * 10004 floats > 16 MiB
    prob, keep = _problem(fq, d)
    U = torch.empty((d.n, d.n), dtype=torch.complex128, device="cuda")
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_build_UT_static(prob, U)
    assert e.value.status == fq.FQ_EINVAL and "floquet_build_UT_static" in fq.floquet_last_error()

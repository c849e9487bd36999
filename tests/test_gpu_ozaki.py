"""FP64 emulation on the tensor cores (FQ_OZAKI: fixed-point BF16 slices, exact FP32 partial
sums) against the FP64 oracle.

Tolerance: the FP64 / emulated-path target, max |U - U_oracle| <= 1e-10.  Six 8-bit slices keep
48 bits of each row's scale and the 21 slice products drop terms below 2^-48 of it, so one
product is good to about 2^-44 of its largest entry; a few hundred products stay far inside
1e-10 (the chains below print their errors, typically 1e-13 .. 1e-12).
"""
import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


def cuda_c128(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def test_ozaki_goe64_build(fq):
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=fq.FQ_OZAKI)
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    u = U.cpu().numpy()
    ref = o.build_ut_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps))
    err = np.max(np.abs(u - ref))
    print(f"GOE64 Ozaki: max err {err:.3e}")
    assert err <= TOL
    mx, fro = fq.api.unitarity_defect(U)
    assert mx <= 1e-12


@pytest.mark.parametrize("n,nc", [(200, 37), (300, 300)])
def test_ozaki_ragged_propagate(fq, n, nc):
    """N = 200 (padded to 256, one partial 128-state tile) and N = 300 (padded to 384, three
    partial tiles), steps 2..9 of 24, a non-even drive, random unit states."""
    M = 24
    h0, h1 = fi.goe(n, 1401), fi.goe(n, 1402)
    drv = fi.Drive(0.2, 1.3, 1.1, 0.6)
    x0 = fi.ginibre(n, 1403)[:nc]
    x0 /= np.linalg.norm(x0, axis=1, keepdims=True)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         precision=fq.FQ_OZAKI)
    X = plan.propagate(cuda_c128(x0), 2, 10).cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    ref = o.propagate_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M), x0.T, 2, 10).T
    err = np.max(np.abs(X - ref))
    print(f"N={n} Ozaki 8 steps: max err {err:.3e}")
    assert err <= TOL


def test_ozaki_magnus6(fq):
    n, M = 40, 16
    h0, h1 = fi.goe(n, 1501), fi.goe(n, 1502)
    drv = fi.Drive(0.2, 1.4, 1.1, 0.5)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         magnus_order=6, precision=fq.FQ_OZAKI)
    U = plan.build_UT().cpu().numpy()
    rp, oms = o.plan_dense6(h0, h1, drv, M)
    assert np.max(np.abs(U - o.build_ut_dense6(rp, oms))) <= TOL


def test_ozaki_matches_fp64_path_and_flags_bounds(fq):
    """Same plan through the plain FP64 kernels and the emulation; caller bounds at 0.4 of the
    true span raise FQ_EBOUND from the emulation's epilogue too."""
    n, M = 130, 12
    h0, h1 = fi.goe(n, 1701), fi.goe(n, 1702)
    kw = dict(omega=1.2, f_ac=0.9, steps=M)
    U64 = fq.Plan.dense(h0, h1, **kw).build_UT().cpu().numpy()
    Uoz = fq.Plan.dense(h0, h1, precision=fq.FQ_OZAKI, **kw).build_UT().cpu().numpy()
    assert np.max(np.abs(U64 - Uoz)) <= TOL
    pm = o.plan_for_drive_dense(h0, h1, fi.Drive(0.0, 0.9, 1.2), M)
    c, w = 0.5 * (pm.e_min + pm.e_max), 0.2 * (pm.e_max - pm.e_min)
    plan = fq.Plan.dense(h0, h1, precision=fq.FQ_OZAKI, e_min=c - w, e_max=c + w, **kw)
    plan.build_UT()
    assert plan.check_status() == fq.FQ_EBOUND


@pytest.mark.slow
def test_ozaki_goe4096_sampled(fq):
    """Dense GOE N = 4096 (seeds 3, 4; A = 2, omega = 2, M = 512): 256 basis states through
    steps 0..7 against the oracle on the same states."""
    m = fi.config_goe4096()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=fq.FQ_OZAKI)
    cols = np.arange(0, 4096, 16)
    x0 = np.zeros((len(cols), 4096), complex)
    x0[np.arange(len(cols)), cols] = 1.0
    X = plan.propagate(cuda_c128(x0), 0, 8).cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    ref = o.propagate_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps), x0.T, 0, 8).T
    err = np.max(np.abs(X - ref))
    print(f"GOE4096 Ozaki 8 steps: max err {err:.3e}")
    assert err <= TOL


@pytest.mark.slow
def test_ozaki_goe4096_full_build_sampled_columns(fq):
    """The dense benchmark workload end to end in FP64 emulation (GOE N = 4096, M = 512): the U_T
    the library builds against the oracle's propagation of 4 sampled basis states through all
    512 steps, and the unitarity defect over 64 columns."""
    import torch
    m = fi.config_goe4096()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=fq.FQ_OZAKI)
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    cols = [0, 1500, 2047, 4095]
    x0 = np.zeros((4096, len(cols)), complex)
    x0[cols, np.arange(len(cols))] = 1.0
    ref = o.propagate_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps), x0)
    err = np.max(np.abs(U[:, cols].cpu().numpy() - ref))
    sample = torch.arange(0, 4096, 64, dtype=torch.int32, device="cuda")
    mx, fro = fq.api.unitarity_defect(U, sample)
    print(f"GOE4096 Ozaki full build: max err {err:.3e}; defect max {mx:.2e} fro {fro:.2e}")
    assert err <= TOL
    assert mx <= 1e-11


@pytest.mark.parametrize("precision", ["FQ_FP64", "FQ_OZAKI", "FQ_BF16X6"])
def test_fixed_chebyshev_terms_match_converged_series(fq, precision):
    """L fixed at 50 (the paper's timing runs) with the 6th-order scheme: past convergence the
    extra terms carry Bessel weights below 1e-30, so U_T equals the oracle's tolerance-truncated
    chain to each path's accuracy."""
    n, M = 48, 16
    h0, h1 = fi.goe(n, 2101), fi.goe(n, 2102)
    drv = fi.Drive(0.2, 1.4, 1.1, 0.5)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         magnus_order=6, cheb_terms=50, precision=getattr(fq, precision))
    assert plan.info.L == 50
    U = plan.build_UT().cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    rp, oms = o.plan_dense6(h0, h1, drv, M)
    err = np.max(np.abs(U - o.build_ut_dense6(rp, oms)))
    print(f"L = 50 {precision}: max err {err:.2e} (oracle L = {rp.L})")
    assert err <= (1e-10 if precision != "FQ_BF16X6" else 1e-5)

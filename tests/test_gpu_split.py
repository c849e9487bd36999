"""Split-precision dense path (tcgen05 BF16 slices, FP32 accumulation) against the FP64 oracle.

Tolerance: max |U - U_oracle| <= min(1e-5, 2 M R eps + 4 sqrt(M L) eps).  1e-5 is the accuracy
target for FP32-level split paths; the second term is the bound of the FP32 tridiagonal path with
eps the relative error of one sliced product:
  * FQ_BF16X3 (2 slices, products hi*hi + hi*lo + lo*hi): a bf16 slice keeps 8 significant bits,
    so two slices represent x to 2^-18 relative, and the dropped lo*lo term is of the same
    size; eps = 2^-17.
  * FQ_BF16X6 (3 slices, 6 products a + b < 3): the representation error is 2^-27, and FP32
    accumulation and the FP32 master copies dominate; eps = 2^-23.
"""
import math

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu

EPS = {2: 2.0 ** -17, 3: 2.0 ** -23}


SPLIT_TARGET = 1e-5


def tol_split(M, L, R, ns):
    e = EPS[ns]
    return min(SPLIT_TARGET, 2.0 * M * R * e + 4.0 * math.sqrt(M * L) * e)


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


def cuda_c128(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


SHAPES = [(2, 2, 64, 0), (2, 2, 64, 32), (3, 3, 64, 0), (2, 2, 128, 0), (3, 3, 128, 0)]  # (prec, NS, width, K stage)


@pytest.mark.parametrize("prec,ns,tile,tk", SHAPES)
def test_split_goe64_build(fq, prec, ns, tile, tk):
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=prec,
                         tile_n=tile, tile_k=tk)
    U = plan.build_UT().cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    ref = o.build_ut_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps))
    err = np.max(np.abs(U - ref))
    tol = tol_split(m.steps, plan.info.L, plan.info.R, ns)
    print(f"GOE64 split NS={ns}: max err {err:.3e} (tol {tol:.3e})")
    assert err <= tol


@pytest.mark.parametrize("prec,ns,tile,tk", SHAPES)
def test_split_ragged_propagate(fq, prec, ns, tile, tk):
    """N = 200 (K' padded to 512, output tiles ragged), 37 states (one partial 128-row tile),
    steps 2..9 of 24, non-even drive."""
    n, M = 200, 24
    h0, h1 = fi.goe(n, 1301), fi.goe(n, 1302)
    drv = fi.Drive(0.2, 1.3, 1.1, 0.6)
    x0 = fi.ginibre(n, 1303)[:37]
    x0 /= np.linalg.norm(x0, axis=1, keepdims=True)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         precision=prec, tile_n=tile, tile_k=tk)
    X = plan.propagate(cuda_c128(x0), 2, 10).cpu().numpy()
    ref = o.propagate_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M), x0.T, 2, 10).T
    err = np.max(np.abs(X - ref))
    assert err <= tol_split(8, plan.info.L, plan.info.R, ns), err


@pytest.mark.slow
def test_split_goe4096_sampled(fq):
    """Dense GOE N = 4096 (seeds 3, 4; A = 2, omega = 2, M = 512), BF16X6: 256 basis states
    through steps 0..7, against the oracle on the same states."""
    import torch
    m = fi.config_goe4096()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=3)
    cols = np.arange(0, 4096, 16)
    x0 = np.zeros((len(cols), 4096), complex)
    x0[np.arange(len(cols)), cols] = 1.0
    X = plan.propagate(cuda_c128(x0), 0, 8).cpu().numpy()
    assert plan.check_status() == fq.FQ_OK
    ref = o.propagate_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps), x0.T, 0, 8).T
    err = np.max(np.abs(X - ref))
    print(f"GOE4096 BF16X6 8 steps: max err {err:.3e}")
    assert err <= tol_split(8, plan.info.L, plan.info.R, 3)


@pytest.mark.slow
@pytest.mark.parametrize("prec,ns", [(2, 2), (3, 3)])
def test_split_goe4096_full_build_sampled_columns(fq, prec, ns):
    """The dense benchmark workload end to end (GOE N = 4096, M = 512, tile 128): the U_T the
    library builds (one call, all 4096 states) against the oracle's propagation of 6 sampled
    basis states through all 512 steps, and the unitarity defect over 64 columns (stated, and
    checked against what the entry bound implies)."""
    import torch
    m = fi.config_goe4096()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=prec)
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    cols = [0, 1, 1000, 2047, 3001, 4095]
    x0 = np.zeros((4096, len(cols)), complex)
    x0[cols, np.arange(len(cols))] = 1.0
    ref = o.propagate_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps), x0)
    got = U[:, cols].cpu().numpy()
    err = np.max(np.abs(got - ref))
    sample = torch.arange(0, 4096, 64, dtype=torch.int32, device="cuda")
    mx, fro = fq.api.unitarity_defect(U, sample)
    print(f"GOE4096 full build NS={ns}: max err {err:.3e} (tol {SPLIT_TARGET:.0e}); defect max {mx:.2e} fro {fro:.2e}")
    assert err <= SPLIT_TARGET
    # U = U_exact + D with |D_ij| <= e gives |(U^+U - 1)_cj| <= 2 sqrt(N) e + N e^2
    e = SPLIT_TARGET
    assert mx <= 2 * math.sqrt(4096) * e + 4096 * e * e

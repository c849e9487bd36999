"""floquet_grad (through the C ABI) against the FP64 oracle's discrete adjoint and against central
finite differences of its own loss.  Both sides freeze the spectral bounds from the same f
(reading R11); the library's Lanczos bounds differ slightly from the oracle's exact ones, which
changes the Chebyshev truncation only at the 1e-14 level, so FP64 gradients agree to 1e-9."""
import math

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


def cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def gpu_grad(fq, h0, h1, w, fm, period, stride, f_plan=None):
    plan = fq.Plan.piecewise(h0, h1, fm if f_plan is None else f_plan, period=period, checkpoint_stride=stride)
    loss, g = plan.grad(cuda(fm), cuda(w.astype(np.complex128)))
    assert plan.check_status() == fq.FQ_OK
    return plan, float(loss.item()), g.cpu().numpy()


@pytest.mark.parametrize("n,M,stride", [(12, 20, 6), (9, 5, 16), (33, 7, 1)])
def test_grad_matches_oracle(fq, n, M, stride):
    """Ragged checkpoint segments (20 = 3*6 + 2), a single segment (M < s) and s = 1."""
    h0, h1 = fi.goe(n, 1101), fi.goe(n, 1102)
    w = fi.haar_unitary(n, 1103)
    fm = 1.0 + 0.1 * fi.normal(1104, M)
    T = 2 * math.pi
    plan, loss, g = gpu_grad(fq, h0, h1, w, fm, T, stride)
    ref_plan = o.plan_piecewise(h0, h1, T, fm)
    ref_loss, ref_g = o.grad_piecewise(h0, h1, w, ref_plan, fm)
    assert abs(loss - ref_loss) <= 1e-12
    assert np.max(np.abs(g - ref_g)) <= 1e-9 * np.max(np.abs(ref_g))


def test_grad_directional_fd(fq):
    """<grad, v> against a central difference of the GPU's own loss along v (FP64, <= 1e-6 rel)."""
    n, M = 64, 32
    h0, h1 = fi.goe(n, 1201), fi.goe(n, 1202)
    w = fi.haar_unitary(n, 1203)
    fm = 1.0 + 0.1 * fi.normal(1204, M)
    v = fi.normal(1205, M)
    T = 2 * math.pi
    # one frozen plan for all three evaluations (bounds must not follow f)
    plan = fq.Plan.piecewise(h0, h1, fm, period=T, checkpoint_stride=8)
    Wd = cuda(w.astype(np.complex128))
    _, g = plan.grad(cuda(fm), Wd)
    d = 1e-5
    lp, _ = plan.grad(cuda(fm + d * v), Wd)
    lm, _ = plan.grad(cuda(fm - d * v), Wd)
    fd = (lp.item() - lm.item()) / (2 * d)
    gv = float(g.cpu().numpy() @ v)
    assert abs(fd - gv) <= 1e-6 * abs(gv)


def test_grad_config5_shape_vs_oracle(fq):
    """The adjoint workload's shape (M = 256 piecewise steps, checkpoints every 16, T = 2 pi) at
    N = 128 so that the oracle finishes in seconds."""
    n, M = 128, 256
    h0, h1 = fi.goe(n, 6), fi.goe(n, 7)
    w = fi.haar_unitary(n, 8)
    fm = 1.0 + 0.1 * fi.normal(9, M)
    T = 2 * math.pi
    plan, loss, g = gpu_grad(fq, h0, h1, w, fm, T, 16)
    ref_plan = o.plan_piecewise(h0, h1, T, fm)
    ref_loss, ref_g = o.grad_piecewise(h0, h1, w, ref_plan, fm)
    assert abs(loss - ref_loss) <= 1e-11
    assert np.max(np.abs(g - ref_g)) <= 1e-9 * np.max(np.abs(ref_g))


def test_grad_argument_errors(fq):
    import torch
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=10)
    f = torch.zeros(10, dtype=torch.float64, device="cuda")
    W = torch.zeros((64, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(fq.FloquetError) as e:
        plan.grad(f, W, ws=torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert e.value.status == fq.FQ_EINVAL

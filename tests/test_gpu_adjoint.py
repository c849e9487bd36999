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


def split_grad_tol(plan, h1, eps, loss):
    """Bound on max_m |dL/df_m - exact| for a split-precision gradient, from the arithmetic:
    the forward and adjoint chains each keep a state's 2-norm error below
    eps_c = 2 M R eps + 4 sqrt(M L) eps (the forward split bound), the dot GEMM adds ~eps, and
    every term |<bbar_l, E psi_{l-1}>| <= ||bbar_l||_F ||E||_2 ||psi_{l-1}||_F with
    ||bbar_l||_F <= ||G||_F sum_j (j+1)|a_j|, ||G||_F = |tau| / N^{3/2} (unitary backward chain,
    |tau| = N sqrt(1 - loss)), ||psi_{l-1}||_F <= sqrt(N); dL/df_m = 2 Re sum of L terms with
    |w_l| <= 2."""
    from scipy.special import jv
    info = plan.info
    M, L, R = info.steps, info.L, info.R
    a = np.array([jv(0, R)] + [2 * jv(k, R) for k in range(1, L + 1)])
    B = float(np.sum((np.arange(L + 1) + 1) * np.abs(a)))
    e_norm = np.max(np.abs(np.linalg.eigvalsh(h1))) / info.delta_e
    eps_c = 2 * M * R * eps + 4 * math.sqrt(M * L) * eps
    term = math.sqrt(max(1.0 - loss, 0.0)) * B * e_norm
    return 4 * L * (2 * eps_c + 2 * eps) * term


@pytest.mark.parametrize("prec,eps", [("BF16X3", 2.0 ** -17), ("BF16X6", 2.0 ** -23)])
@pytest.mark.parametrize("n,M,stride,tile", [(40, 20, 6, 64), (200, 12, 5, 128), (130, 9, 16, 64)])
def test_split_grad_matches_oracle(fq, prec, eps, n, M, stride, tile):
    """Tensor-core gradient (BF16 slices, FP32 accumulation) against the FP64 oracle: ragged
    tiles (40, 130, 200 rows in 128-row tiles), ragged checkpoint segments and a single segment."""
    h0, h1 = fi.goe(n, 1301), fi.goe(n, 1302)
    w = fi.haar_unitary(n, 1303)
    fm = 1.0 + 0.1 * fi.normal(1304, M)
    T = 2 * math.pi
    plan = fq.Plan.piecewise(h0, h1, fm, period=T, checkpoint_stride=stride, precision=getattr(fq, "FQ_" + prec),
                             tile_n=tile)
    loss, g = plan.grad(cuda(fm), cuda(w.astype(np.complex128)))
    assert plan.check_status() == fq.FQ_OK
    g = g.cpu().numpy()
    ref_plan = o.plan_piecewise(h0, h1, T, fm)
    ref_loss, ref_g = o.grad_piecewise(h0, h1, w, ref_plan, fm)
    tol = split_grad_tol(plan, h1, eps, ref_loss)
    err = np.max(np.abs(g - ref_g))
    print(f"split grad {prec} n={n}: max err {err:.2e} (tol {tol:.2e}, max |g| {np.max(np.abs(ref_g)):.2e})")
    assert err <= tol
    assert abs(float(loss.item()) - ref_loss) <= 4 * (2 * M * plan.info.R * eps + 4 * math.sqrt(M * plan.info.L) * eps)


def test_split_grad_config5_shape_vs_oracle(fq):
    """The adjoint workload's shape (M = 256, checkpoints every 16) at N = 128, BF16X3."""
    n, M = 128, 256
    h0, h1 = fi.goe(n, 6), fi.goe(n, 7)
    w = fi.haar_unitary(n, 8)
    fm = 1.0 + 0.1 * fi.normal(9, M)
    T = 2 * math.pi
    plan = fq.Plan.piecewise(h0, h1, fm, period=T, checkpoint_stride=16, precision=fq.FQ_BF16X3)
    loss, g = plan.grad(cuda(fm), cuda(w.astype(np.complex128)))
    assert plan.check_status() == fq.FQ_OK
    ref_plan = o.plan_piecewise(h0, h1, T, fm)
    ref_loss, ref_g = o.grad_piecewise(h0, h1, w, ref_plan, fm)
    err = np.max(np.abs(g.cpu().numpy() - ref_g))
    tol = split_grad_tol(plan, h1, 2.0 ** -17, ref_loss)
    print(f"split grad config-5 shape: max err {err:.2e} (tol {tol:.2e}, max |g| {np.max(np.abs(ref_g)):.2e})")
    assert err <= tol


def test_fidelity_loss_autograd(fq):
    """fidelity_loss as a torch.autograd.Function: backward returns the library's adjoint scaled by
    the cotangent (chain rule through 3 L + sum f), and <grad, v> matches a central difference of
    the differentiable loss itself (FP64, <= 1e-6 relative)."""
    import torch
    n, M = 48, 24
    h0, h1 = fi.goe(n, 1401), fi.goe(n, 1402)
    w = fi.haar_unitary(n, 1403)
    fm = 1.0 + 0.1 * fi.normal(1404, M)
    v = fi.normal(1405, M)
    plan = fq.Plan.piecewise(h0, h1, fm, period=2 * math.pi, checkpoint_stride=5)
    W = cuda(w.astype(np.complex128))
    f = cuda(fm).requires_grad_(True)
    loss = fq.fidelity_loss(plan, f, W)
    (3.0 * loss + f.sum()).backward()
    _, g = plan.grad(cuda(fm), W)
    assert torch.allclose(f.grad, 3.0 * g + 1.0, rtol=0, atol=1e-15)
    d = 1e-5
    with torch.no_grad():
        lp = fq.fidelity_loss(plan, cuda(fm + d * v), W).item()
        lm = fq.fidelity_loss(plan, cuda(fm - d * v), W).item()
    gv = float(g.cpu().numpy() @ v)
    assert abs((lp - lm) / (2 * d) - gv) <= 1e-6 * abs(gv)


# ------------------------------------------------------------------ FP64 emulation (FQ_OZAKI)
@pytest.mark.parametrize("n,M,stride", [(12, 20, 6), (33, 7, 1), (200, 12, 5), (130, 9, 16)])
def test_ozaki_grad_matches_oracle(fq, n, M, stride):
    """Gradient with every product in FP64 emulation on the tensor cores against the FP64 oracle,
    held to the FP64 criterion (1e-9 of max |g|, loss to 1e-11): ragged tiles, ragged checkpoint
    segments, s = 1 and a single segment."""
    h0, h1 = fi.goe(n, 1901), fi.goe(n, 1902)
    w = fi.haar_unitary(n, 1903)
    fm = 1.0 + 0.1 * fi.normal(1904, M)
    T = 2 * math.pi
    plan = fq.Plan.piecewise(h0, h1, fm, period=T, checkpoint_stride=stride, precision=fq.FQ_OZAKI)
    loss, g = plan.grad(cuda(fm), cuda(w.astype(np.complex128)))
    assert plan.check_status() == fq.FQ_OK
    g = g.cpu().numpy()
    ref_plan = o.plan_piecewise(h0, h1, T, fm)
    ref_loss, ref_g = o.grad_piecewise(h0, h1, w, ref_plan, fm)
    err = np.max(np.abs(g - ref_g))
    print(f"Ozaki grad n={n}: max err {err:.2e} (max |g| {np.max(np.abs(ref_g)):.2e}), "
          f"loss err {abs(float(loss.item()) - ref_loss):.1e}")
    assert abs(float(loss.item()) - ref_loss) <= 1e-11
    assert err <= 1e-9 * np.max(np.abs(ref_g))


def test_ozaki_grad_matches_fp64_path(fq):
    """N = 512, M = 32: the emulated gradient against the plain FP64 GPU gradient (1e-9 of max |g|)."""
    n, M = 512, 32
    h0, h1 = fi.goe(n, 2001), fi.goe(n, 2002)
    w = cuda(fi.haar_unitary(n, 2003).astype(np.complex128))
    fm = 1.0 + 0.1 * fi.normal(2004, M)
    T = 2 * math.pi
    p64 = fq.Plan.piecewise(h0, h1, fm, period=T, checkpoint_stride=16)
    poz = fq.Plan.piecewise(h0, h1, fm, period=T, checkpoint_stride=16, precision=fq.FQ_OZAKI)
    l64, g64 = p64.grad(cuda(fm), w)
    loz, goz = poz.grad(cuda(fm), w)
    g64, goz = g64.cpu().numpy(), goz.cpu().numpy()
    print(f"Ozaki vs FP64 grad n=512: {np.max(np.abs(goz - g64)):.2e} (max |g| {np.max(np.abs(g64)):.2e})")
    assert abs(l64.item() - loz.item()) <= 1e-11
    assert np.max(np.abs(goz - g64)) <= 1e-9 * np.max(np.abs(g64))


def test_ozaki_grad_directional_fd(fq):
    """<grad, v> against a central difference of the emulated loss along v (<= 1e-6 relative), at
    the size of the FP64 finite-difference test (the gradient shrinks like 1/N, and at N = 512 the
    loss's own rounding divided by the step would already reach the criterion)."""
    n, M = 64, 32
    h0, h1 = fi.goe(n, 1201), fi.goe(n, 1202)
    w = cuda(fi.haar_unitary(n, 1203).astype(np.complex128))
    fm = 1.0 + 0.1 * fi.normal(1204, M)
    v = fi.normal(1205, M)
    plan = fq.Plan.piecewise(h0, h1, fm, period=2 * math.pi, checkpoint_stride=8, precision=fq.FQ_OZAKI)
    _, g = plan.grad(cuda(fm), w)
    d = 1e-5
    lp, _ = plan.grad(cuda(fm + d * v), w)
    lm, _ = plan.grad(cuda(fm - d * v), w)
    fd = (lp.item() - lm.item()) / (2 * d)
    gv = float(g.cpu().numpy() @ v)
    assert abs(fd - gv) <= 1e-6 * abs(gv)


# ------------------------------------------------------------------ the gradient workload at its size
@pytest.mark.slow
@pytest.mark.parametrize("prec", ["FQ_FP64", "FQ_OZAKI", "FQ_BF16X3", "FQ_BF16X6"])
def test_grad_config5_full_size_vs_stored_oracle(fq, prec):
    """The gate-fidelity workload at its own size (GOE N = 1024, seeds 6-9, M = 256 piecewise
    steps, T = 2 pi, checkpoints every 16) against the oracle's loss and gradient, computed once
    by tests/golden/make_golden.py adjoint1024 (oracle only).  FP64 and the FP64 emulation are
    held to 1e-9 of max |g| and the loss to 1e-11; the split precisions to their arithmetic bound
    (split_grad_tol) with the loss to the forward split bound."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    ref = mg.read_adjoint("adjoint1024.txt")
    ref_g = np.array(ref["g"])
    a = fi.config_adjoint()
    assert a.h0.shape[0] == 1024 and len(a.f) == 256 == len(ref_g)
    plan = fq.Plan.piecewise(a.h0, a.h1, a.f, period=a.period, checkpoint_stride=16, precision=getattr(fq, prec))
    assert plan.info.L == int(ref["L"])
    loss, g = plan.grad(cuda(a.f), cuda(a.target.astype(np.complex128)))
    assert plan.check_status() == fq.FQ_OK
    g = g.cpu().numpy()
    err = np.max(np.abs(g - ref_g))
    lerr = abs(float(loss.item()) - ref["loss"])
    print(f"config-5 gradient {prec}: max err {err:.2e} (max |g| {np.max(np.abs(ref_g)):.2e}), loss err {lerr:.1e}")
    if prec in ("FQ_FP64", "FQ_OZAKI"):
        assert lerr <= 1e-11
        assert err <= 1e-9 * np.max(np.abs(ref_g))
    else:
        eps = 2.0 ** -17 if prec == "FQ_BF16X3" else 2.0 ** -23
        assert err <= split_grad_tol(plan, a.h1, eps, ref["loss"])
        M, R, L = plan.info.steps, plan.info.R, plan.info.L
        assert lerr <= 4 * (2 * M * R * eps + 4 * math.sqrt(M * L) * eps)

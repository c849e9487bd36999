"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (written here, derived in the design notes):
  * FP64 paths: max |U - U_oracle| <= 1e-10 (the method's own truncation is 1e-14 per step).
  * FP32 tridiagonal paths: max |U - U_oracle| <= tol_f32(M, L, R) = 2 M R u + 4 sqrt(M) L u,
    u = 2^-24.  First term: the FP32 rounding of Omega~'s entries (|entries| <= 1, so
    ||dOmega~||_2 <= 2u) perturbs each step's exponent exp(-i R Omega~) by at most 2Ru, and that
    systematic error adds up coherently over M steps.  Second term: the rounding of the L
    operator products of a step (about L u per step on a unit-norm state) adds up as a random
    walk over M unitary steps (factor 4 of headroom).  Both bound a column's 2-norm error and so
    its largest entry error.  Every FP32 check is also held to the 1e-5 accuracy target of
    FP32-level paths: the test tolerance is min(1e-5, that bound).
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def f32_bound(M, L, R):
    """2 M R u + 4 sqrt(M) L u: the FP32 rounding bound of a column's 2-norm error."""
    return 2.0 * M * R * U32 + 4.0 * math.sqrt(M) * L * U32


def tol_f32(M, L, R):
    """Entry tolerance of FP32 paths: the 2-norm bound, capped at the FP32-level target 1e-5."""
    return min(1e-5, f32_bound(M, L, R))


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1508_07621_gb300 as fq
    return fq


def to_np(t):
    return t.detach().cpu().numpy()


def cuda_c128(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


# ------------------------------------------------------------------ dense FP64
def test_goe64_fp64_build(fq):
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps)
    assert plan.info.L == 7
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    ref_plan = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    ref = o.build_ut_dense(m.h0, m.h1, ref_plan)
    u = to_np(U)
    assert np.max(np.abs(u - ref)) <= 1e-10
    assert np.max(np.abs(u - u.T)) <= 1e-12          # even drive: U_T = U_T^T
    mx, fro = fq.api.unitarity_defect(U)
    assert mx <= 1e-12 and fro <= 1e-12
    eps, eps_ref = o.quasienergies(u, m.drive.period), o.quasienergies(ref, m.drive.period)
    assert np.max(np.abs(eps - eps_ref)) <= 1e-10


def test_dense_fp64_ragged_propagate_range(fq):
    """N = 37 (ragged against the 32/8 tiles), 5 random states, steps 3..10 of 16, non-even drive."""
    n, M = 37, 16
    h0, h1 = fi.goe(n, 801), fi.goe(n, 802)
    drv = fi.Drive(0.3, 1.4, 1.1, 0.8)
    x0 = fi.ginibre(n, 803)[:5]
    x0 /= np.linalg.norm(x0, axis=1, keepdims=True)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M)
    X = plan.propagate(cuda_c128(x0), 3, 11)
    ref = o.propagate_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M), x0.T, 3, 11).T
    assert np.max(np.abs(to_np(X) - ref)) <= 1e-10
    # empty range copies, zero states is a no-op
    Y = plan.propagate(cuda_c128(x0), 4, 4)
    assert np.array_equal(to_np(Y), x0)


@pytest.mark.parametrize("precision", ["FQ_FP64", "FQ_DF32", "FQ_OZAKI"])
@pytest.mark.parametrize("n,scale", [(1, 1.0), (2, 1.0), (6, 1e-9)])
def test_dense_fp64_degenerate(fq, n, scale, precision):
    """N = 1 (zero spectral width), N = 2, and a tiny operator with L = 1 (one-term steps), on the
    FP64 path and the two emulated ones."""
    h0, h1 = scale * fi.goe(n, 901), scale * fi.goe(n, 902)
    drv = fi.Drive(0.1, 0.7, 1.0, 0.2)
    plan = fq.Plan.dense(h0, h1, omega=1.0, f_ac=0.7, f_dc=0.1, phi0=0.2, steps=12,
                         precision=getattr(fq, precision))
    if scale < 1e-6:
        assert plan.info.L == 1
    U = to_np(plan.build_UT())
    ref = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, 12))
    assert np.max(np.abs(U - ref)) <= 1e-10


# ------------------------------------------------------------------ tridiagonal
def dimer_plan(fq, d, precision, kernel=0):
    return fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=d.drive.omega, f_ac=d.drive.f_ac,
                           f_dc=d.drive.f_dc, phi0=d.drive.phi0, steps=d.steps, precision=precision,
                           kernel=kernel)


@pytest.mark.parametrize("precision,kernel", [(0, 1), (1, 1), (1, 2), (0, 3), (1, 3), (4, 3), (4, 0)])
def test_dimer40_all_paths(fq, precision, kernel):
    """Small dimer (dim 41, M = 100): FP64 / FP32 streaming, FP32 resident, FP64 / FP32 tiled,
    double-float tiled (explicit and by AUTO)."""
    d = fi.config_dimer(nb=40, steps=100)
    plan = dimer_plan(fq, d, precision, kernel)
    U = to_np(plan.build_UT())
    assert plan.check_status() == fq.FQ_OK
    ref = o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag,
                             o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps))
    tol = tol_f32(d.steps, plan.info.L, plan.info.R) if precision == 1 else 1e-10
    assert np.max(np.abs(U - ref)) <= tol


@pytest.mark.parametrize("nb", [4, 2047, 6000, 10239])
def test_dimer_resident_ragged_sizes(fq, nb):
    """Resident kernel across its per-thread widths (4..20 rows) and ragged tails; 3 states,
    20 steps of the M = 2000 chain (phase offset drive)."""
    d = fi.config_dimer(nb=nb, steps=2000)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = dimer_plan(fq, d, 1, 2)
    n = d.n
    x0 = np.zeros((3, n), complex)
    x0[0, 0] = 1
    x0[1, n - 1] = 1
    x0[2] = fi.ginibre(n, 11)[0] if n < 4000 else np.exp(2j * np.pi * fi.uniform(12, n))
    x0[2] /= np.linalg.norm(x0[2])
    X = to_np(plan.propagate(cuda_c128(x0), 0, 20))
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    ref = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x0.T, 0, 20).T
    assert np.max(np.abs(X - ref)) <= tol_f32(20, plan.info.L, plan.info.R)


def _oracle_dimer_column(j):
    d = fi.config_dimer()
    p = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    return o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag, p, [j])[:, 0]


@pytest.mark.slow
def test_dimer_full_size_resident_sampled_columns(fq):
    """The benchmarked workload (dim 10001, M = 2000, L = 39, FP32 resident kernel, one launch
    over all 10001 states): sampled columns against the oracle, unitarity on 64 columns."""
    import torch
    cols = [0, 1, 5000, 9999, 10000]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(cols)) as pool:
        pending = pool.map_async(_oracle_dimer_column, cols)
        d = fi.config_dimer()
        plan = dimer_plan(fq, d, 1, 0)
        assert plan.info.L == 39
        U = plan.build_UT()
        assert plan.check_status() == fq.FQ_OK
        ref = np.stack(pending.get(timeout=1800), axis=1)
    got = to_np(U[:, cols])
    tol = tol_f32(d.steps, 39, plan.info.R)
    err = np.max(np.abs(got - ref))
    print(f"dimer 10001 FP32 resident: max err {err:.3e} (tol {tol:.3e})")
    assert err <= tol
    sample = torch.arange(0, d.n, 157, dtype=torch.int32, device="cuda")
    mx, fro = fq.api.unitarity_defect(U, sample)
    # (U^+ U - 1)[c][j] = <u_c|du_j> + <du_c|u_j> + ...: twice a column's 2-norm error
    assert mx <= 2 * f32_bound(d.steps, 39, plan.info.R)


def test_dimer_u0_full_size_closed_form(fq):
    """U = 0 dimer at dim 10001 (FP32 resident, one launch over all states): H is the nb-boson
    image of h = [[f/2, -1], [-1, -f/2]], so U_T = D(u) with u the 2x2 Magnus chain of exact
    exponentials (closed form, no oracle).  Checks: U_T maps the SU(2) coherent state
    c_n = sqrt(C(nb, n)) a^n b^(nb-n) to the coherent state of u (a, b), and Tr U_T equals the
    character sum_k l1^k l2^(nb-k)."""
    import torch
    from scipy.special import gammaln
    nb = 10000
    d = fi.config_dimer(nb=nb, U=0.0)
    plan = dimer_plan(fq, d, 1, 0)
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    h = d.drive.period / d.steps
    sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    u = np.eye(2, dtype=complex)
    for m in range(d.steps):
        tau = (m + 0.5) * h
        f = d.drive.f_ac * math.cos(d.drive.omega * tau)
        f1 = -d.drive.f_ac * d.drive.omega * math.sin(d.drive.omega * tau)
        f2 = -d.drive.f_ac * d.drive.omega ** 2 * math.cos(d.drive.omega * tau)
        b = h * f + h ** 3 * f2 / 24
        c = h ** 3 * f1 / 12
        # omega = a h0 + b h1 + c i[h0,h1] with h0 = -sigma_x, h1 = sigma_z / 2, i[h0,h1] = -sigma_y
        w = np.array([-h, -c, 0.5 * b])
        r = np.linalg.norm(w)
        u = (math.cos(r) * np.eye(2) - 1j * math.sin(r) / r * sum(wi * s for wi, s in zip(w, sig))) @ u
    tol = f32_bound(d.steps, plan.info.L, plan.info.R)   # 2-norm errors of whole states below

    def coherent(a, b):
        n = np.arange(nb + 1)
        logc = 0.5 * (gammaln(nb + 1) - gammaln(n + 1) - gammaln(nb - n + 1)) + n * np.log(a + 0j) \
            + (nb - n) * np.log(b + 0j)
        return np.exp(logc)

    a0, b0 = math.cos(0.55), np.exp(0.3j) * math.sin(0.55)
    c0 = coherent(a0, b0)
    a1, b1 = u @ np.array([a0, b0])
    got = to_np(U @ cuda_c128(c0))
    err = np.linalg.norm(got - coherent(a1, b1))
    print(f"U=0 dimer coherent-state error {err:.3e} (tol {tol:.3e})")
    assert err <= tol
    l1, l2 = np.linalg.eigvals(u)
    k = np.arange(nb + 1)
    char = np.sum(np.exp(-1j * (k * -np.angle(l1) + (nb - k) * -np.angle(l2))))
    assert abs(complex(U.diagonal().sum().item()) - char) <= math.sqrt(d.n) * tol


def test_bound_violation_sets_status(fq):
    """Host-made fault: caller bounds at half the true half-span put Omega~'s spectrum in
    [-2, 2]; with R ~ 11 the truncated series is no longer unitary.  The device checks must
    report FQ_EBOUND (no trap), and the status clears for the next call."""
    d = fi.config_dimer(nb=40, steps=10)
    p = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    c, w = 0.5 * (p.e_min + p.e_max), 0.25 * (p.e_max - p.e_min)
    for precision, kernel in ((0, 1), (1, 1), (1, 2)):
        plan = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=3.0, f_ac=1.5, steps=d.steps,
                               precision=precision, kernel=kernel, e_min=c - w, e_max=c + w)
        plan.build_UT()
        assert plan.check_status() == fq.FQ_EBOUND, (precision, kernel)
        assert plan.check_status() == fq.FQ_OK
    m = fi.config_goe64()
    pm = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    c, w = 0.5 * (pm.e_min + pm.e_max), 0.2 * (pm.e_max - pm.e_min)
    for kernel in (fq.FQ_KERNEL_RESIDENT, fq.FQ_KERNEL_TILED):
        plan = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=m.steps, e_min=c - w, e_max=c + w,
                             kernel=kernel)
        plan.build_UT()
        assert plan.check_status() == fq.FQ_EBOUND, kernel


def test_workspace_errors(fq):
    import torch
    d = fi.config_dimer(nb=40, steps=10)
    plan = dimer_plan(fq, d, 1, 1)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    U = torch.empty((d.n, d.n), dtype=torch.complex128, device="cuda")
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_build_UT(plan.handle, U, small)
    assert e.value.status == fq.FQ_EINVAL
    with pytest.raises(fq.FloquetError):
        fq.floquet_propagate(plan.handle, U, U, d.n, 5, 3, small)


@pytest.mark.parametrize("precision,kernel", [(1, 2), (1, 1), (0, 1)])
def test_paper_dimer_parameters(fq, precision, kernel):
    """The paper's own dimer (v = 1, U nb = 2, (U/2)(n1 - n2)^2, H_mod = n2 - n1, f = 2.7 +
    2.5 cos 3t) at nb = 1000, M = 1000 (R = 11.1, L = 34): 4 states through steps 3..27 against
    the oracle, on the resident and streaming FP32 kernels and the streaming FP64 kernel."""
    d = fi.config_dimer_paper(nb=1000, steps=1000)
    plan = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=d.drive.omega, f_ac=d.drive.f_ac,
                           f_dc=d.drive.f_dc, steps=d.steps, precision=precision, kernel=kernel)
    assert plan.info.L == 34
    n = d.n
    x0 = np.zeros((4, n), complex)
    x0[0, 0] = 1
    x0[1, n // 2] = 1
    x0[2, n - 1] = 1
    x0[3] = fi.ginibre(n, 2101)[0]
    x0[3] /= np.linalg.norm(x0[3])
    X = to_np(plan.propagate(cuda_c128(x0), 3, 28))
    assert plan.check_status() == fq.FQ_OK
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    ref = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x0.T, 3, 28).T
    tol = 1e-10 if precision == 0 else tol_f32(25, plan.info.L, plan.info.R)
    assert np.max(np.abs(X - ref)) <= tol


@pytest.mark.parametrize("precision,nb,m_end", [(0, 3000, 6), (1, 3000, 6), (0, 10000, 3), (1, 12000, 3),
                                                 (0, 2011, 4), (0, 2012, 4), (4, 3000, 6), (4, 10000, 3)])
def test_dimer_tiled_kernel_segments(fq, precision, nb, m_end):
    """Tiled chain (one launch per step, L halo rows a side): several segments with a ragged tail
    (dim 3001, 10001), FP32 beyond the resident kernel's 10240 rows (dim 12001), and dims at one
    segment and one past it (2012 and 2013 rows: 2048-row tiles at L = 18); first, middle and last basis
    states and a random unit vector, steps 1..m_end-1 of the M = 2000 chain (phase offset drive)."""
    d = fi.config_dimer(nb=nb, steps=2000)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = dimer_plan(fq, d, precision, 3)
    n = d.n
    x0 = np.zeros((4, n), complex)
    x0[0, 0] = 1
    x0[1, n // 2] = 1
    x0[2, n - 1] = 1
    x0[3] = np.exp(2j * np.pi * fi.uniform(2201, n))
    x0[3] /= np.linalg.norm(x0[3])
    X = to_np(plan.propagate(cuda_c128(x0), 1, m_end))
    assert plan.check_status() == fq.FQ_OK
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    ref = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x0.T, 1, m_end).T
    tol = tol_f32(m_end - 1, plan.info.L, plan.info.R) if precision == 1 else 1e-10
    assert np.max(np.abs(X - ref)) <= tol


def test_tiled_kernel_rejects_long_series(fq):
    """L above 128 (one step over a whole period of the dim-1001 dimer) is refused, not run."""
    d = fi.config_dimer(nb=1000, steps=1)
    prob, keep = fq.make_problem(d.n, fq.FQ_TRIDIAG, d.h0_diag, d.h1_diag, d.drive.period, d.steps, h0_off=d.h0_off,
                                 f_ac=1.5, omega=3.0, precision=fq.FQ_FP64, kernel=fq.FQ_KERNEL_TILED)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_plan_create(prob)
    assert e.value.status == fq.FQ_EUNSUPPORTED


@pytest.mark.slow
def test_dimer_full_size_double_float_sampled_columns(fq):
    """The benchmark dimer (dim 10001, M = 2000, L = 39) built in double-float on the tiled kernel:
    sampled columns against the FP64 oracle at the FP64 tolerance 1e-10."""
    cols = [0, 5000, 10000]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(cols)) as pool:
        pending = pool.map_async(_oracle_dimer_column, cols)
        d = fi.config_dimer()
        plan = dimer_plan(fq, d, fq.FQ_DF32, 0)
        U = plan.build_UT()
        assert plan.check_status() == fq.FQ_OK
        ref = np.stack(pending.get(timeout=1800), axis=1)
    err = np.max(np.abs(to_np(U[:, cols]) - ref))
    print(f"dimer 10001 double-float tiled: max err {err:.3e}")
    assert err <= 1e-10


@pytest.mark.parametrize("case", ["resident", "tiled64", "dense64", "split3"])
def test_column_slices_bitwise_and_deterministic(fq, case):
    """Columns of U_T are independent (one state per unit of work): U_T built in one call equals,
    bit for bit, the propagation of the identity in three uneven slices of states, and a second
    build equals the first bit for bit."""
    import torch
    if case in ("resident", "tiled64"):
        d = fi.config_dimer(nb=700, steps=60)
        plan = dimer_plan(fq, d, 1 if case == "resident" else 0, 2 if case == "resident" else 3)
        n = d.n
    else:
        n = 200
        h0, h1 = fi.goe(n, 2301), fi.goe(n, 2302)
        plan = fq.Plan.dense(h0, h1, omega=1.3, f_ac=1.1, steps=12, precision=0 if case == "dense64" else fq.FQ_BF16X3)
    U = plan.build_UT()
    U2 = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    assert torch.equal(U, U2)
    eye = torch.eye(n, dtype=torch.complex128, device="cuda")
    cuts = [0, 37, n // 2 + 5, n]
    for a, b in zip(cuts, cuts[1:]):
        X = plan.propagate(eye[a:b].contiguous())          # rows = states a..b-1
        assert torch.equal(X.transpose(0, 1), U[:, a:b])


@pytest.mark.parametrize("precision,kernel", [(1, 2), (5, 4), (0, 1)])
def test_build_report(fq, precision, kernel):
    """floquet_build_UT_report: the same U_T as floquet_build_UT bit for bit, the plan's L, R and
    bounds, a unitarity defect at the path's level over sampled columns and a positive device time;
    a bad column count is refused."""
    import torch
    d = fi.config_dimer(nb=300, steps=200)
    plan = dimer_plan(fq, d, precision, kernel)
    ref = plan.build_UT()
    U = torch.empty_like(ref)
    ws = fq.workspace(plan.workspace_size())
    rep = fq.floquet_build_UT_report(plan.handle, U, ws, 32)
    assert torch.equal(U, ref)
    info = plan.info
    assert rep.L == info.L and rep.R == info.R and rep.e_min == info.e_min and rep.e_max == info.e_max
    assert rep.beta == info.beta and rep.delta_e == info.delta_e and rep.defect_columns == 32
    assert rep.defect_max <= (2 * f32_bound(d.steps, info.L, info.R) if precision == 1 else 1e-10)
    assert 0 < rep.defect_fro <= rep.defect_max * math.sqrt(d.n) and rep.build_ms > 0
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_build_UT_report(plan.handle, U, ws, d.n + 1)
    assert e.value.status == fq.FQ_EINVAL


@pytest.mark.parametrize("case", ["resident", "dfl", "dense64", "split"])
def test_column_blocks_assemble_build_UT(fq, case):
    """floquet_build_UT_columns (one rank's share of the column split, §5): the uneven blocks a
    2- or 3-rank split gives, written into their slots of one gather buffer, are U_T in
    column-major order, bit for bit the single-call build; out-of-range blocks are refused."""
    import torch
    from paper_1508_07621_gb300 import shard
    if case in ("resident", "dfl"):
        d = fi.config_dimer(nb=700, steps=40)
        plan = dimer_plan(fq, d, 1 if case == "resident" else 4, 2 if case == "resident" else 3)
        n = d.n
    else:
        n = 130
        h0, h1 = fi.goe(n, 2401), fi.goe(n, 2402)
        plan = fq.Plan.dense(h0, h1, omega=1.3, f_ac=1.1, steps=10, precision=0 if case == "dense64" else fq.FQ_BF16X3)
    U = plan.build_UT()
    for world in (2, 3):
        buf = torch.full((world * -(-n // world), n), float("nan"), dtype=torch.complex128, device="cuda")
        ws = fq.workspace(fq.floquet_columns_workspace_size(plan.handle, -(-n // world)))
        for r in range(world):
            j0, j1, _ = shard.column_block(n, r, world)
            if j1 > j0:
                fq.floquet_build_UT_columns(plan.handle, j0, j1 - j0, shard.slot(buf, r, world), ws)
        assert plan.check_status() == fq.FQ_OK
        assert torch.equal(buf[:n].transpose(0, 1), U)
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_build_UT_columns(plan.handle, n - 2, 3, buf, ws)
    assert e.value.status == fq.FQ_EINVAL


# ------------------------------------------------------------------ dense FP64, resident kernel
@pytest.mark.parametrize("n", [1, 5, 32, 33, 64, 65, 100, 128])
def test_dense_fp64_resident_kernel(fq, n):
    """The small-N resident chain (clusters of ceil(N/32) CTAs, 64 steps per launch) against the
    oracle and against the per-term kernel: ragged row blocks (33, 65, 100), one to four CTAs per
    state, M = 70 crossing a launch boundary, a non-even drive."""
    M = 70
    h0, h1 = fi.goe(n, 1101), fi.goe(n, 1102)
    drv = fi.Drive(0.2, 1.3, 1.7, 0.4)
    kw = dict(omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M)
    res = fq.Plan.dense(h0, h1, kernel=fq.FQ_KERNEL_RESIDENT, **kw)
    til = fq.Plan.dense(h0, h1, kernel=fq.FQ_KERNEL_TILED, **kw)
    U, V = res.build_UT(), til.build_UT()
    assert res.check_status() == fq.FQ_OK and til.check_status() == fq.FQ_OK
    ref = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M))
    assert np.max(np.abs(to_np(U) - ref)) <= 1e-10
    assert np.max(np.abs(to_np(U) - to_np(V))) <= 1e-12


def test_dense_fp64_resident_segments_and_limits(fq):
    """Steps 50..139 of 150 (two launch boundaries inside the range) on 7 states, against the
    oracle; N = 129 cannot take the resident kernel when it is asked for."""
    n, M = 48, 150
    h0, h1 = fi.goe(n, 1201), fi.goe(n, 1202)
    drv = fi.Drive(0.0, 1.0, 1.0, 0.3)
    x0 = fi.ginibre(n, 1203)[:7]
    x0 /= np.linalg.norm(x0, axis=1, keepdims=True)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, phi0=drv.phi0, steps=M,
                         kernel=fq.FQ_KERNEL_RESIDENT)
    X = plan.propagate(cuda_c128(x0), 50, 140)
    ref = o.propagate_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M), x0.T, 50, 140).T
    assert np.max(np.abs(to_np(X) - ref)) <= 1e-10
    with pytest.raises(fq.FloquetError) as e:
        fq.Plan.dense(fi.goe(129, 1), fi.goe(129, 2), omega=1.0, f_ac=1.0, steps=4, kernel=fq.FQ_KERNEL_RESIDENT)
    assert e.value.status == fq.FQ_EUNSUPPORTED


@pytest.mark.parametrize("n", [1, 5, 33, 64, 100, 128])
def test_dense_double_float_resident(fq, n):
    """FQ_DF32 on the dense resident chain (double-float arithmetic on the FP32 pipes, FP64
    states): against the oracle at the FP64 / emulated target, M = 70 across a launch boundary,
    a non-even drive."""
    M = 70
    h0, h1 = fi.goe(n, 1101), fi.goe(n, 1102)
    drv = fi.Drive(0.2, 1.3, 1.7, 0.4)
    plan = fq.Plan.dense(h0, h1, omega=drv.omega, f_ac=drv.f_ac, f_dc=drv.f_dc, phi0=drv.phi0, steps=M,
                         precision=fq.FQ_DF32)
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    ref = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, drv, M))
    err = np.max(np.abs(to_np(U) - ref))
    print(f"dense double-float resident N={n}: max err {err:.3e}")
    assert err <= 1e-10


def test_dense_double_float_limits_and_bounds(fq):
    """Dense FQ_DF32 needs the resident kernel (N <= 128); caller bounds at 0.4 of the true span
    raise FQ_EBOUND from its device check."""
    for n, kernel in ((129, fq.FQ_KERNEL_AUTO), (64, fq.FQ_KERNEL_TILED)):
        with pytest.raises(fq.FloquetError) as e:
            fq.Plan.dense(fi.goe(n, 1), fi.goe(n, 2), omega=1.0, f_ac=1.0, steps=4, precision=fq.FQ_DF32,
                          kernel=kernel)
        assert e.value.status == fq.FQ_EUNSUPPORTED
    m = fi.config_goe64()
    pm = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    c, w = 0.5 * (pm.e_min + pm.e_max), 0.2 * (pm.e_max - pm.e_min)
    plan = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=m.steps, e_min=c - w, e_max=c + w,
                         precision=fq.FQ_DF32)
    plan.build_UT()
    assert plan.check_status() == fq.FQ_EBOUND


def test_bounded_wait_timeout_is_reported(fq):
    """Failure detection without a fault: a wait on an mbarrier that nothing arrives on gives up
    after its cycle limit and records the timeout; the host reads FQ_ETIMEOUT once, the word is
    cleared, and the context and the plan keep working."""
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=4)
    fq.floquet_selftest_wait(plan.handle, 2_000_000)
    assert plan.check_status() == fq.FQ_ETIMEOUT
    assert plan.check_status() == fq.FQ_OK
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    mx, _ = fq.api.unitarity_defect(U)
    assert mx <= 1e-12
    with pytest.raises(fq.FloquetError) as e:
        fq.floquet_selftest_wait(plan.handle, 0)
    assert e.value.status == fq.FQ_EINVAL

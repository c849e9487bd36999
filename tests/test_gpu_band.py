"""The tridiagonal chain on the tensor cores in FP64 emulation (FQ_OZAKI on a tridiagonal plan, the
band kernel): parity with the FP64 oracle at the FP64 criterion (max |U - U_oracle| <= 1e-10)
through the C ABI, on the small dimer's whole U_T, ragged sizes (one to many 64-row operator
blocks, 128-state tiles with a ragged tail), L up to the kernel's limit of 47, the benchmark
dimer at full size (sampled columns), and the bitwise column split."""
import math
import multiprocessing as mp

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


def to_np(t):
    return t.detach().cpu().numpy()


def cuda_c128(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def band_plan(fq, d, kernel=0):
    return fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=d.drive.omega, f_ac=d.drive.f_ac,
                           f_dc=d.drive.f_dc, phi0=d.drive.phi0, steps=d.steps, precision=fq.FQ_OZAKI,
                           kernel=kernel)


@pytest.mark.parametrize("kernel", [0, 4])
def test_band_dimer40_whole_UT(fq, kernel):
    """dim 41 (one 64-row block, one 128-state tile), M = 100: U_T by AUTO and by the explicit
    band kernel against the oracle, and unitary to FP64 level."""
    d = fi.config_dimer(nb=40, steps=100)
    plan = band_plan(fq, d, kernel)
    U = to_np(plan.build_UT())
    assert plan.check_status() == fq.FQ_OK
    ref = o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag,
                             o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps))
    err = np.max(np.abs(U - ref))
    print(f"band dimer40: max err {err:.2e}")
    assert err <= 1e-10
    assert np.max(np.abs(U.conj().T @ U - np.eye(d.n))) <= 1e-10   # the FP64 criterion, on U^+ U - 1


@pytest.mark.parametrize("nb,steps,m_end", [(4, 2000, 4), (63, 2000, 4), (64, 2000, 4), (700, 2000, 6),
                                            (2047, 2000, 5), (10000, 2000, 3), (10000, 1480, 3)])
def test_band_ragged_sizes(fq, nb, steps, m_end):
    """First, middle and last basis states and two random unit vectors (5 states in one ragged
    128-state tile) through steps 1 .. m_end-1 of the chain with a phase-offset drive: 5 to 10001
    rows (one to 157 operator blocks), L from 4 to 47 (M = 1480 at dim 10001)."""
    d = fi.config_dimer(nb=nb, steps=steps)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = band_plan(fq, d)
    assert plan.info.L <= 47
    n = d.n
    x0 = np.zeros((5, n), complex)
    x0[0, 0] = 1
    x0[1, n // 2] = 1
    x0[2, n - 1] = 1
    for r, seed in ((3, 2501), (4, 2502)):
        x0[r] = np.exp(2j * np.pi * fi.uniform(seed, n)) * (1.0 + fi.uniform(seed + 10, n))
        x0[r] /= np.linalg.norm(x0[r])
    X = to_np(plan.propagate(cuda_c128(x0), 1, m_end))
    assert plan.check_status() == fq.FQ_OK
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    assert refp.L == plan.info.L
    ref = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x0.T, 1, m_end).T
    err = np.max(np.abs(X - ref))
    print(f"band nb={nb} M={steps} L={plan.info.L}: max err {err:.2e}")
    assert err <= 1e-10


def test_band_refocusing_states_take_the_rescaling_path(fq):
    """States that refocus: x0 = P_0^+ P_1^+ y with y = (e_a + e_b + e_c) / sqrt(3) (three basis
    vectors far apart), so X_0 = P_1^+ y spreads over three bands of about 2L + 1 components and
    X_1 = y.  The product cuts X_1 into the next step's slices at the scale X_0's largest |Re| or
    |Im| predicts, one bit up: 2^(floor(log2 a) + 3) for a maximum a, which holds values up to
    2^(floor(log2 a) + 2).  With a < 1/4 (checked on the oracle's X_0) that is at most 1/2, below
    y's 1/sqrt(3), so those states are flagged and cut again from the double-float states at their
    exact scale.  Three refocusing states and two plain ones (dim 701, 6 steps) against the oracle
    at the FP64 criterion, and X_1 against y."""
    d = fi.config_dimer(nb=700, steps=200)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = band_plan(fq, d)
    n = d.n
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    prop = lambda x, m0, m1: o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x, m0, m1)
    eye = np.eye(n, dtype=complex)
    p0, p1 = prop(eye, 0, 1), prop(eye, 1, 2)
    y = np.zeros((n, 3), complex)
    for c, ks in enumerate(((50, 300, 550), (100, 350, 600), (150, 400, 650))):
        y[list(ks), c] = 1.0 / np.sqrt(3.0)
    x_0 = p1.conj().T @ y                           # X_0 of the refocusing states
    part_max = lambda v: np.max(np.maximum(np.abs(v.real), np.abs(v.imag)), axis=0)
    assert np.all(part_max(x_0) < 0.25) and np.all(part_max(y) > 0.5)
    x0 = np.concatenate([p0.conj().T @ x_0, np.zeros((n, 2), complex)], axis=1)
    x0[0, 3] = 1.0
    x0[:, 4] = np.exp(2j * np.pi * fi.uniform(2601, n)) / np.sqrt(n)
    X1 = to_np(plan.propagate(cuda_c128(x0.T), 0, 2))
    assert plan.check_status() == fq.FQ_OK
    assert np.max(np.abs(X1[:3] - y.T)) <= 1e-10
    X = to_np(plan.propagate(cuda_c128(x0.T), 0, 6))
    ref = prop(x0, 0, 6).T
    err = np.max(np.abs(X - ref))
    print(f"band refocusing states: max err {err:.2e}")
    assert err <= 1e-10


def test_band_next_band_formed_inside_the_product(fq):
    """4096 states (the product then forms the next step's band in its own warps): the dim-701
    dimer (L = 32, 11 operator blocks, 88 blocks of 8 band rows spread over the persistent CTAs),
    random unit states through 3 steps, every state against the oracle."""
    d = fi.config_dimer(nb=700, steps=200)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = band_plan(fq, d)
    n, nc = d.n, 4096
    x0 = np.exp(2j * np.pi * fi.uniform(2701, n * nc)).reshape(n, nc) * (1.0 + fi.uniform(2702, n * nc).reshape(n, nc))
    x0 /= np.linalg.norm(x0, axis=0)
    X = to_np(plan.propagate(cuda_c128(x0.T), 1, 4))
    assert plan.check_status() == fq.FQ_OK
    refp = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    ref = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, refp, x0, 1, 4).T
    err = np.max(np.abs(X - ref))
    print(f"band 4096 states, next band in the product: max err {err:.2e}")
    assert err <= 1e-10


def test_band_propagation_captured_in_a_cuda_graph(fq):
    """The band path on a capturing stream: floquet_propagate of 4096 states (so the product also
    forms the next band) through 3 steps, captured in a CUDA graph and replayed twice, equals the
    direct call bit for bit."""
    import torch
    d = fi.config_dimer(nb=700, steps=200)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)
    plan = band_plan(fq, d)
    n, nc = d.n, 4096
    x0 = np.exp(2j * np.pi * fi.uniform(2801, n * nc)).reshape(nc, n) / np.sqrt(n)
    X0 = cuda_c128(x0)
    ws = fq.workspace(plan.workspace_size(nc))
    ref = torch.empty_like(X0)
    fq.floquet_propagate(plan.handle, X0, ref, nc, 1, 4, ws)
    torch.cuda.synchronize()
    out = torch.empty_like(X0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fq.floquet_propagate(plan.handle, X0, out, nc, 1, 4, ws)
    for _ in range(2):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert plan.check_status() == fq.FQ_OK


def test_band_many_state_tiles_and_column_split(fq):
    """dim 701 (11 operator blocks), all 701 states (6 state tiles, ragged): U_T equals the column
    blocks of a 3-rank split bit for bit, and matches the oracle."""
    import torch
    from paper_1508_07621_gb300 import shard
    d = fi.config_dimer(nb=700, steps=200)    # L = 32
    plan = band_plan(fq, d)
    n = d.n
    U = plan.build_UT()
    assert plan.check_status() == fq.FQ_OK
    buf = torch.full((3 * -(-n // 3), n), float("nan"), dtype=torch.complex128, device="cuda")
    ws = fq.workspace(fq.floquet_columns_workspace_size(plan.handle, -(-n // 3)))
    for r in range(3):
        j0, j1, _ = shard.column_block(n, r, 3)
        fq.floquet_build_UT_columns(plan.handle, j0, j1 - j0, shard.slot(buf, r, 3), ws)
    assert torch.equal(buf[:n].transpose(0, 1), U)
    cols = [0, 1, 350, 699, 700]
    ref = o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag,
                             o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps), cols)
    assert np.max(np.abs(to_np(U[:, cols]) - ref)) <= 1e-10


def test_band_kernel_selection(fq):
    """FQ_OZAKI tridiagonal plans run on the band kernel only; it refuses other precisions and
    series longer than its window (L > 47: 40 steps of the dim-701 dimer give L = 85)."""
    d = fi.config_dimer(nb=40, steps=100)
    for prec, kern in ((fq.FQ_FP32, fq.FQ_KERNEL_BAND), (fq.FQ_OZAKI, fq.FQ_KERNEL_TILED),
                       (fq.FQ_OZAKI, fq.FQ_KERNEL_RESIDENT)):
        with pytest.raises(fq.FloquetError) as e:
            fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=3.0, f_ac=1.5, steps=100, precision=prec,
                            kernel=kern)
        assert e.value.status == fq.FQ_EUNSUPPORTED
    d = fi.config_dimer(nb=700, steps=40)
    with pytest.raises(fq.FloquetError) as e:
        band_plan(fq, d)
    assert e.value.status == fq.FQ_EUNSUPPORTED


def test_kernel_timing_records_the_step_kernel(fq):
    """floquet_kernel_timing: a band build of M = 100 steps records 100 launches of k_oz_band whose
    summed event time lies inside the build's own; reading clears the record; switched off,
    nothing is recorded; an FP32 build records its one resident launch."""
    import torch
    d = fi.config_dimer(nb=40, steps=100)
    stream = torch.cuda.current_stream()
    U = torch.empty((d.n, d.n), dtype=torch.complex128, device="cuda")
    plan = band_plan(fq, d)
    ws = fq.workspace(plan.workspace_size())
    fq.floquet_kernel_timing(plan.handle, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fq.floquet_build_UT(plan.handle, U, ws, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launches, ms, name = fq.floquet_kernel_time(plan.handle)
    assert (launches, name) == (100, "k_oz_band")
    assert 0.0 < ms <= e0.elapsed_time(e1)
    assert fq.floquet_kernel_time(plan.handle) == (0, 0.0, "")
    fq.floquet_kernel_timing(plan.handle, False)
    fq.floquet_build_UT(plan.handle, U, ws, stream)
    assert fq.floquet_kernel_time(plan.handle)[0] == 0
    p32 = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=d.drive.omega, f_ac=d.drive.f_ac,
                          steps=d.steps, precision=fq.FQ_FP32)
    fq.floquet_kernel_timing(p32.handle, True)
    fq.floquet_build_UT(p32.handle, U, fq.workspace(p32.workspace_size()), stream)
    launches, ms, name = fq.floquet_kernel_time(p32.handle)
    assert (launches, name) == (1, "k_tri_resident") and ms > 0.0


def _oracle_dimer_column(j):
    d = fi.config_dimer()
    p = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    return o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag, p, [j])[:, 0]


@pytest.mark.slow
def test_band_full_size_sampled_columns(fq):
    """The benchmark dimer (dim 10001, M = 2000, L = 39) on the band kernel, the bench's launch
    configuration (floquet_build_UT over all 10001 states): sampled columns against the oracle at
    the FP64 criterion, unitarity on 64 columns."""
    import torch
    cols = [0, 1, 5000, 9999, 10000]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(cols)) as pool:
        pending = pool.map_async(_oracle_dimer_column, cols)
        d = fi.config_dimer()
        plan = band_plan(fq, d)
        assert plan.info.L == 39
        U = plan.build_UT()
        assert plan.check_status() == fq.FQ_OK
        ref = np.stack(pending.get(timeout=1800), axis=1)
    err = np.max(np.abs(to_np(U[:, cols]) - ref))
    print(f"band dimer 10001: max err {err:.3e}")
    assert err <= 1e-10
    sample = torch.arange(0, d.n, 157, dtype=torch.int32, device="cuda")
    mx, fro = fq.api.unitarity_defect(U, sample)
    assert mx <= 1e-10

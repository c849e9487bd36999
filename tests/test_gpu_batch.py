"""Batched scan (one CUDA graph over many plans) and the tile autotuner."""
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


def test_batch_matches_individual_builds(fq):
    """Mixed scan (split X3 of several sizes, FP64 dense, FP64 emulation, double-float dense, FP32
    resident tridiagonal) as one graph
    on 3 lanes: every output equals the same plan's own floquet_build_UT bit for bit (the kernels
    are deterministic), and one instance equals the oracle within the split tolerance."""
    import torch
    insts = fi.batch_scan(count=5, seed=77, n_lo=40, n_hi=300)
    plans = [fq.Plan.dense(fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1), omega=s.omega, f_ac=s.amplitude,
                           steps=12, precision=fq.FQ_BF16X3) for s in insts]
    plans.append(fq.Plan.dense(fi.goe(48, 5001), fi.goe(48, 5002), omega=1.0, f_ac=1.0, steps=10))
    # the emulated paths: tensor-core FP64 emulation and the double-float resident chain
    plans.append(fq.Plan.dense(fi.goe(150, 5003), fi.goe(150, 5004), omega=1.0, f_ac=1.0, steps=6,
                               precision=fq.FQ_OZAKI))
    plans.append(fq.Plan.dense(fi.goe(70, 5005), fi.goe(70, 5006), omega=1.0, f_ac=1.0, steps=9,
                               precision=fq.FQ_DF32))
    d = fi.config_dimer(nb=40, steps=20)
    plans.append(fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=3.0, f_ac=1.5, steps=20))
    outs = [torch.empty((p.n, p.n), dtype=torch.complex128, device="cuda") for p in plans]
    handles = [p.handle for p in plans]
    ws = fq.workspace(fq.floquet_batch_workspace_size(handles))
    b = fq.floquet_batch_create(handles, outs, ws, 3)
    try:
        fq.floquet_batch_launch(b)
        torch.cuda.synchronize()
        for p, u in zip(plans, outs):
            ref = p.build_UT()
            assert torch.equal(u, ref)
        # replay: same results again
        for u in outs:
            u.zero_()
        fq.floquet_batch_launch(b)
        torch.cuda.synchronize()
        for p, u in zip(plans, outs):
            assert torch.equal(u, p.build_UT())
    finally:
        fq.floquet_batch_destroy(b)
    s = insts[0]
    h0, h1 = fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1)
    ref = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, fi.Drive(0.0, s.amplitude, s.omega), 12))
    eps = 2.0 ** -17
    tol = min(1e-5, 2 * 12 * plans[0].info.R * eps + 4 * math.sqrt(12 * plans[0].info.L) * eps)  # split target
    assert np.max(np.abs(outs[0].cpu().numpy() - ref)) <= tol


def test_autotune_picks_a_tile_and_stays_correct(fq):
    m = fi.config_goe64()
    plan = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=m.steps, precision=fq.FQ_BF16X3)
    tile = plan.autotune()
    assert tile in (64, 128)
    U = plan.build_UT().cpu().numpy()
    ref = o.build_ut_dense(m.h0, m.h1, o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps))
    eps = 2.0 ** -17   # BF16X3: hi + lo slices carry 16 bits
    tol = min(1e-5, 2 * m.steps * plan.info.R * eps + 4 * math.sqrt(m.steps * plan.info.L) * eps)  # split target
    assert np.max(np.abs(U - ref)) <= tol
    p64 = fq.Plan.dense(m.h0, m.h1, omega=1.0, f_ac=1.0, steps=10)
    assert p64.autotune() == 0   # FP64 path: nothing to tune

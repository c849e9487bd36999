"""The batched-scan workload at its full size, in the launch configuration bench.py times, against
the FP64 oracle on sampled outputs.  (Named to run after the other GPU files.)"""
import math

import numpy as np
import pytest

import floquet_inputs as fi
import oracle as o

pytestmark = pytest.mark.gpu

SPLIT_TARGET = 1e-5
STEPS = 256


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


@pytest.mark.slow
def test_full_scan_sampled_against_oracle(fq):
    """48 GOE instances (N ~ U{256..2048}, omega ~ U[0.5, 4], A ~ U[0.5, 3], M = 256), BF16X3
    with autotuned tiles, built by one persistent launch over (instance, step, term, tile) work
    units (lanes = 0, as bench.py times it): the smallest, the median and the
    largest instance each against the oracle's propagation of 3 basis states (first, middle and
    last) through all 256 steps, to the split target; every instance's unitarity defect over 16
    columns within what that target implies (|(U^+U - 1)_cj| <= 2 sqrt(N) e + N e^2)."""
    import torch
    insts = fi.batch_scan()
    models = [(fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1), fi.Drive(0.0, s.amplitude, s.omega)) for s in insts]
    plans = [fq.Plan.dense(h0, h1, omega=d.omega, f_ac=d.f_ac, steps=STEPS, precision=fq.FQ_BF16X3)
             for h0, h1, d in models]
    ws1 = fq.workspace(max(p.workspace_size() for p in plans))
    tiles = [p.autotune(ws1) for p in plans]
    assert all(t in (64, 128) for t in tiles)
    del ws1
    outs = [torch.empty((p.n, p.n), dtype=torch.complex128, device="cuda") for p in plans]
    handles = [p.handle for p in plans]
    ws = fq.workspace(fq.floquet_batch_workspace_size(handles))
    b = fq.floquet_batch_create(handles, outs, ws, 0)
    try:
        fq.floquet_batch_launch(b)
        torch.cuda.synchronize()
    finally:
        fq.floquet_batch_destroy(b)
    assert all(p.check_status() == fq.FQ_OK for p in plans)
    e = SPLIT_TARGET
    for u in outs:
        n = u.shape[0]
        cols = torch.arange(0, n, max(1, n // 16), dtype=torch.int32, device="cuda")[:16]
        mx, _ = fq.api.unitarity_defect(u, cols)
        assert mx <= 2 * math.sqrt(n) * e + n * e * e, (n, mx)
    order = np.argsort([s.n for s in insts], kind="stable")
    for i in (order[0], order[len(order) // 2], order[-1]):
        h0, h1, d = models[i]
        n = h0.shape[0]
        cols = [0, n // 2, n - 1]
        x0 = np.zeros((n, len(cols)), complex)
        x0[cols, np.arange(len(cols))] = 1.0
        ref = o.propagate_dense(h0, h1, o.plan_for_drive_dense(h0, h1, d, STEPS), x0)
        err = float(np.max(np.abs(outs[i][:, cols].cpu().numpy() - ref)))
        print(f"scan instance {i}: N = {n}, L = {plans[i].info.L}, tile {tiles[i]}, max err {err:.3e}")
        assert err <= SPLIT_TARGET, (n, err)

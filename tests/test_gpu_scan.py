"""The batched scan as one persistent launch (floquet_batch_create with lanes = 0, csrc/scan.cu):
every instance's U_T against the same plan's own floquet_build_UT, bit for bit (both run the same
slices, tile shape, MMA order and epilogue), over ragged sizes, odd and even series lengths L
and scans of 1 to 8 steps; the fall-back to the lane graph for plans the scan does not take; and
one instance against the oracle."""
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


def _models(count=6, seed=91, n_lo=20, n_hi=400):
    """Instances of the scan's recipe at small sizes (N from 150 to 389: one to four 128-state
    blocks, none a multiple of 128), plus a 7-level system (one tile, fewer states than a block
    of 16 output rows)."""
    out = [(fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1), fi.Drive(0.0, s.amplitude, s.omega))
           for s in fi.batch_scan(count=count, seed=seed, n_lo=n_lo, n_hi=n_hi)]
    out.append((fi.goe(7, 7001), fi.goe(7, 7002), fi.Drive(0.0, 1.3, 2.1)))
    return out


def _plans(fq, models, steps, precision, tile_n):
    return [fq.Plan.dense(h0, h1, omega=d.omega, f_ac=d.f_ac, steps=steps, precision=precision, tile_n=tile_n)
            for h0, h1, d in models]


def _scan(fq, plans, lanes=0, launches=2):
    """Runs the batch `launches` times (outputs poisoned with NaN before each) and returns the
    outputs of the last launch."""
    import torch
    outs = [torch.empty((p.n, p.n), dtype=torch.complex128, device="cuda") for p in plans]
    handles = [p.handle for p in plans]
    ws = fq.workspace(fq.floquet_batch_workspace_size(handles))
    b = fq.floquet_batch_create(handles, outs, ws, lanes)
    try:
        for _ in range(launches):
            for u in outs:
                u.fill_(float("nan"))
            fq.floquet_batch_launch(b)
            torch.cuda.synchronize()
            assert all(p.check_status() == fq.FQ_OK for p in plans)
    finally:
        fq.floquet_batch_destroy(b)
    return outs


@pytest.mark.parametrize("precision,tile_n", [("FQ_BF16X3", 64), ("FQ_BF16X3", 128), ("FQ_BF16X6", 64),
                                              ("FQ_BF16X6", 128)])
def test_scan_matches_individual_builds(fq, precision, tile_n):
    """Seven instances (L from 10 to 20, both parities, so the master and left-operand buffers
    rotate both ways) over 8 steps: each U_T from the persistent launch equals the plan's own
    build bit for bit, on the second of two launches of the graph (the counters start again)."""
    import torch
    plans = _plans(fq, _models(), 8, getattr(fq, precision), tile_n)
    Ls = [p.info.L for p in plans]
    assert {L % 2 for L in Ls} == {0, 1} and max(Ls) <= 32
    outs = _scan(fq, plans)
    for p, u in zip(plans, outs):
        assert torch.equal(u, p.build_UT()), (p.n, p.info.L)


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_scan_short_scans(fq, steps):
    """Scans of 1 to 3 steps (no step reuses an Omega~ buffer before the third; the B units of
    the step after the last are skipped): bit for bit the plans' own builds."""
    import torch
    plans = _plans(fq, _models(count=3, seed=92), steps, fq.FQ_BF16X3, 128)
    outs = _scan(fq, plans, launches=1)
    for p, u in zip(plans, outs):
        assert torch.equal(u, p.build_UT()), (p.n, steps)


def test_scan_takes_one_instance_and_matches_the_oracle(fq):
    """A batch of one: the persistent launch against the FP64 oracle, to the split target."""
    h0, h1, d = _models(count=1, seed=93)[0]
    steps = 12
    plan = _plans(fq, [(h0, h1, d)], steps, fq.FQ_BF16X3, 0)[0]
    u = _scan(fq, [plan], launches=1)[0].cpu().numpy()
    ref = o.build_ut_dense(h0, h1, o.plan_for_drive_dense(h0, h1, d, steps))
    eps = 2.0 ** -17
    tol = min(1e-5, 2 * steps * plan.info.R * eps + 4 * math.sqrt(steps * plan.info.L) * eps)  # split target
    assert np.max(np.abs(u - ref)) <= tol


def test_scan_falls_back_to_lanes_for_other_plans(fq):
    """lanes = 0 with a plan the persistent scan does not take (plain FP64 dense): the lane graph
    runs instead, with the same results as the plans' own builds."""
    import torch
    plans = _plans(fq, _models(count=2, seed=94), 6, fq.FQ_BF16X3, 0)
    plans.append(fq.Plan.dense(fi.goe(40, 5101), fi.goe(40, 5102), omega=1.0, f_ac=1.0, steps=6))
    outs = _scan(fq, plans, launches=1)
    for p, u in zip(plans, outs):
        assert torch.equal(u, p.build_UT())

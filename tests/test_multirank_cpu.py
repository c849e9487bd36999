"""The N > 1 paths of bench.py on CPU with gloo ranks on 127.0.0.1 (no GPU involved).

Column split (§5, Fig. 2; the distribute and gather parts of Algorithm 1): every rank takes its
block of U_T's columns from paper_1508_07621_gb300.shard, fills its slot of the gather buffer with
those columns - here from the FP64 oracle, the stand-in for floquet_build_UT_columns - and one
in-place all-gather assembles U_T.  The gathered result must equal the one-rank oracle U_T on
an uneven split (41 columns over 2 ranks), and the job time is the max over ranks.

Replicas (weak scaling): rank r takes its own drive amplitude."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1508_07621_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _dimer():
    import floquet_inputs as fi
    d = fi.config_dimer(nb=40, steps=30)
    d.drive = fi.Drive(0.2, 1.5, 3.0, 0.4)   # phase offset: U_T is not symmetric
    return d


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as o
    d = _dimer()
    plan = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    j0, j1, bs = shard.column_block(d.n, rank, world)
    buf = shard.gather_buffer(d.n, world, device="cpu")
    buf.fill_(float("nan"))                 # nothing but the gather may fill other ranks' slots
    mine = shard.slot(buf, rank, world)
    cols = o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag, plan, list(range(j0, j1)))
    mine[: j1 - j0] = torch.from_numpy(np.ascontiguousarray(cols.T))
    ut_colmajor = shard.all_gather_columns(buf, d.n, dist)
    value, total = bench.job_throughput(1.0 + rank, 3, dist)   # rank r pretends to take 1 + r s
    out[rank] = (j0, j1, bs, ut_colmajor.numpy().copy(), value, total,
                 bench.rank_drive_amplitude(1.5, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_column_split_equals_one_rank():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    import oracle as o
    d = _dimer()
    plan = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    ref = o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag, plan)
    (a0, b0, s0, u0, v0, t0, amp0), (a1, b1, s1, u1, v1, t1, amp1) = out[0], out[1]
    assert (a0, b0, a1, b1, s0) == (0, 21, 21, 41, 21)        # uneven: 21 + 20 columns
    assert np.array_equal(u0, u1)                            # every rank holds the same U_T
    assert np.max(np.abs(u0.T - ref)) == 0.0                 # exactly the one-rank result
    assert t0 == t1 == 2.0                                   # max over ranks
    assert v0 == v1 == world * 3 / 2.0
    assert amp0 == 1.5 and abs(amp1 - 1.51) < 1e-15         # replicas: independent amplitudes


@pytest.mark.parametrize("n", [1, 5, 41, 10001])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_column_blocks_cover_every_column_once(n, world):
    seen = []
    for r in range(world):
        j0, j1, bs = shard.column_block(n, r, world)
        assert 0 <= j0 <= j1 <= n and j1 - j0 <= bs == -(-n // world)
        assert j0 == min(r * bs, n)            # each block starts at its slot
        seen.extend(range(j0, j1))
    assert seen == list(range(n))


def test_column_block_rejects_bad_split():
    for args in [(10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            shard.column_block(*args)

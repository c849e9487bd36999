"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) each take their own drive
amplitude (independent problems, weak scaling) and the job time is the max over ranks.  Each
rank also checks that its problem is the benchmark workload with only eps1 changed, by running
the FP64 oracle on two states for two steps of its own chain (no GPU involved)."""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import floquet_inputs as fi
    import oracle as o
    amp = bench.rank_drive_amplitude(1.5, rank)
    # each rank: a slice of its own chain with the oracle (stand-in for the GPU build)
    d = fi.config_dimer(nb=60, steps=40)
    drv = fi.Drive(0.0, amp, 3.0)
    plan = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, drv, d.steps)
    x0 = np.zeros((d.n, 2), complex)
    x0[0, 0] = x0[d.n - 1, 1] = 1.0
    x = o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, plan, x0, 0, 2)
    local_seconds = 1.0 + rank          # pretend rank r took 1 + r seconds
    value, total = bench.job_throughput(local_seconds, 3, dist)
    out[rank] = (amp, value, total, float(np.linalg.norm(x[:, 0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (a0, v0, t0, n0), (a1, v1, t1, n1) = out[0], out[1]
    assert a0 == 1.5 and abs(a1 - 1.51) < 1e-15          # independent problems per rank
    assert t0 == t1 == 2.0                                # max over ranks
    assert v0 == v1 == world * 3 / 2.0                   # whole-job U_T/s
    assert abs(n0 - 1.0) < 1e-12 and abs(n1 - 1.0) < 1e-12

"""Benchmark: U_T builds per second on the Bose-Hubbard dimer with nb = 10^4 bosons
(dim 10001, tridiagonal Fock basis), M = 2000 Magnus-4 steps per period, Chebyshev truncated at
|J_{L+1}(R)| < 1e-14 (L = 39), in FP64-level arithmetic by default (--precision df32: the
double-float tiled chain), with the FP32 resident kernel timed beside it (the line's "fp32" key;
--precision fp32 makes it the headline).

One step = one U_T build (the full 10001 x 10001 identity propagated over the period).
N > 1 (torchrun): by default the ranks split each U_T's columns (§5: column blocks propagate
independently, one all-gather assembles U_T; "scaling": "strong"); --shard replicas instead gives
every rank its own drive amplitude (independent problems, "scaling": "weak").

--impl reference times the FP64 CPU oracle on this host on a bounded sample of the same
workload (a few states over a slice of the period) and reports the same metric.

--workload goe4096 (dense GOE N = 4096, M = 512: U_T builds/s) and --workload adjoint (the
gate-fidelity gradient at N = 1024, M = 256: gradients/s), with --precision x3 | x6 | ozaki
(| fp64 for the gradient), print the same contract for the metric's other parts.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NB = 10000
STEPS = 2000
FLOPS_PER_ELEMENT_TERM = 26   # complex tridiagonal apply 18 + recurrence 4 + Bessel accumulation 4
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM traffic of the resident kernel from one ncu capture of `--ncu-case resident` (152 states,
# steps 0..19, k_tri_resident<256, 40>, the current kernel with its L2 prefetch): bytes read, of
# which the 152 initial states are a fixed part; the rest is the per-step (2d, 2e') and rotation
# stream, which grows with waves x steps.  A build also writes U_T once.
RES_NCU = {"read": 28515072.0, "x0": 152 * 10001 * 16, "states": 152, "steps": 20}
RES_TRAFFIC_NOTE = ("per-wave-step coefficient reads of one ncu capture (profiles/k_tri_resident_dimer10001.md) "
                    "x waves x steps, plus the 16 N^2 bytes of U_T")


def resident_traffic(n, steps, states):
    """DRAM bytes of one resident launch over `states` states, scaled from the capture."""
    per_wave_step = (RES_NCU["read"] - RES_NCU["x0"]) / RES_NCU["steps"]
    return per_wave_step * (states / RES_NCU["states"]) * steps + 16.0 * n * states
# double-float tiled chain: FP32 lane operations per element-term (4 complex double-float FMAs of
# 15 packed FP32x2 operations each)
DFL_LANE_OPS_PER_ELEMENT_TERM = 120
# The paper's Table 1 (M = 100, L = 50, 6th order): seconds of Chebyshev iterations for one U_T
# on one node (2 x 8-core Xeon E5-2660, FP64 MKL zgemm), by N.
PAPER_TABLE1_CHEB_S = {256: 4.3, 512: 25.3, 1024: 177.3, 2048: 1296.6, 4096: 9730.5, 5120: 18667.2,
                       10240: 181722.3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-extra", action="store_true",
                    help="dimer: skip the FP32 resident timing reported beside an FP64-level headline")
    ap.add_argument("--fp32-steps", type=int, default=3, help="dimer: timed FP32 resident builds beside the headline")
    ap.add_argument("--shard", choices=["columns", "replicas"], default="columns",
                    help="dimer under torchrun: split each U_T's columns over the ranks with one all-gather "
                         "(default), or give every rank its own drive amplitude")
    ap.add_argument("--workload", choices=["dimer", "dimer-paper", "goe4096", "adjoint", "paper-table1", "batch"],
                    default="dimer",
                    help="dimer: nb = 10^4, J = 1, U nb = 2, f = 1.5 cos 3t, M = 2000 (default); "
                         "dimer-paper: the paper's parameters (U/2)(n1 - n2)^2, f = 2.7 + 2.5 cos 3t, M = 8000; "
                         "goe4096: dense GOE N = 4096 (seeds 3, 4), A = 2, omega = 2, M = 512, U_T builds/s; "
                         "adjoint: gate-fidelity gradient, GOE N = 1024 (seeds 6-9), M = 256, s = 16, grads/s; "
                         "paper-table1: the paper's timing run (GOE N = 4096 with unit-variance entries, "
                         "f = cos(pi t), M = 100, L = 50, 6th order), compared with its Table 1 time; "
                         "batch: a scan of 48 dense GOE instances (N ~ U{256..2048}, omega ~ U[0.5, 4], "
                         "A ~ U[0.5, 3], M = 256) as one CUDA graph over 8 lanes, instances/s")
    ap.add_argument("--n", type=int, default=4096, choices=sorted(PAPER_TABLE1_CHEB_S),
                    help="paper-table1: the matrix size (the rows of the paper's Table 1)")
    ap.add_argument("--lanes", type=int, default=0,
                    help="batch: 0 = one persistent launch over work units (split precisions), 1-32 = a graph of "
                         "per-instance builds on that many branches")
    ap.add_argument("--precision", choices=["x3", "x6", "ozaki", "fp64", "fp32", "df32"], default=None,
                    help="goe4096 / adjoint / batch: BF16X3 (default), BF16X6, FQ_OZAKI (FP64 emulation) or FP64 "
                         "(adjoint only); dimer: ozaki (band kernel on the tensor cores, FP64-level; default), "
                         "df32 (double-float tiled, FP64-level) or fp32 (resident)")
    ap.add_argument("--ncu-case", choices=["resident", "stream", "split", "tile", "dfl", "band", "adjoint", "ozaki",
                                           "dense-resident", "ozaki-grad", "scan"],
                    default=None,
                    help="run one small capture case of a kernel twice and exit (for ncu --set full)")
    return ap.parse_args()


def run_ncu_case(case):
    """Small cases for detailed ncu captures (a few GB at most, inputs larger than L2):
    resident: 152 states (one wave on 152 SMs) over steps 0..19 of the benchmark chain;
    stream:   2048 states through step 0 (39 streaming FP32 term launches, 0.5 GB of states);
    split:    dense GOE N = 4096 (seeds 3, 4), BF16X3 tensor-core terms of step 0 on the identity;
    tile:     2048 states through step 0 on the FP64 tiled kernel (0.65 GB of states);
    dfl:      2048 states through step 0 on the double-float tiled kernel (FQ_DF32, 0.65 GB);
    band:     4096 states through steps 0..2 on the band kernel (FQ_OZAKI, in place: 0.66 GB of
              states, 1.3 GB of double-float states and 2 GB of slices in the workspace; at 4096
              states each product also forms the next step's band, as at the full 10001)
    adjoint:  the BF16X3 gradient at N = 1024 (seeds 6-9) over the first 16 of its 256 steps;
    ozaki-grad: the same in FP64 emulation (FQ_OZAKI);
    ozaki:    dense GOE N = 2048 (seeds 3, 4; A = 2, omega = 2, M = 64), FQ_OZAKI terms of step 0 on
              the identity (0.25 GB of slices, 0.2 GB of FP64 states);
    dense-resident: GOE N = 64 (seeds 1, 2), M = 200, the FP64 resident chain (4 launches);
    scan:     the batched scan's recipe at 6 instances of N in [256, 1024] (seed 5), M = 8, BF16X3
              with 128-row tiles, as one persistent launch (about 0.4 GB of workspace)."""
    import math
    import torch
    import floquet_inputs as fi
    import paper_1508_07621_gb300 as fq
    if case in ("adjoint", "ozaki-grad"):
        n, M = 1024, 16
        fm = 1.0 + 0.1 * fi.normal(9, 256)[:M]
        plan = fq.Plan.piecewise(fi.goe(n, 6), fi.goe(n, 7), fm, period=2 * math.pi * M / 256,
                                 checkpoint_stride=16, tile_n=64,
                                 precision=fq.FQ_BF16X3 if case == "adjoint" else fq.FQ_OZAKI)
        W = torch.tensor(fi.haar_unitary(n, 8), dtype=torch.complex128, device="cuda")
        f = torch.tensor(fm, device="cuda")
        for _ in range(2):
            plan.grad(f, W)
        torch.cuda.synchronize()
        print(f"ncu case {case}: status {plan.check_status()}")
        return
    if case in ("ozaki", "dense-resident"):
        m = fi.config_goe4096(2048, 64) if case == "ozaki" else fi.config_goe64()
        prec = fq.FQ_OZAKI if case == "ozaki" else fq.FQ_FP64
        plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps, precision=prec)
        n = m.n
        x0 = torch.eye(n, dtype=torch.complex128, device="cuda")
        x = torch.empty_like(x0)
        ws = fq.workspace(plan.workspace_size(n))
        for _ in range(2):
            fq.floquet_propagate(plan.handle, x0, x, n, 0, 1 if case == "ozaki" else m.steps, ws)
        torch.cuda.synchronize()
        print(f"ncu case {case}: status {plan.check_status()}, L = {plan.info.L}")
        return
    if case == "scan":
        insts = fi.batch_scan(count=6, seed=5, n_lo=256, n_hi=1024)
        plans = [fq.Plan.dense(fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1), omega=s.omega, f_ac=s.amplitude,
                               steps=8, precision=fq.FQ_BF16X3, tile_n=128) for s in insts]
        outs = [torch.empty((p.n, p.n), dtype=torch.complex128, device="cuda") for p in plans]
        handles = [p.handle for p in plans]
        ws = fq.workspace(fq.floquet_batch_workspace_size(handles))
        b = fq.floquet_batch_create(handles, outs, ws, 0)
        try:
            for _ in range(2):
                fq.floquet_batch_launch(b)
            torch.cuda.synchronize()
        finally:
            fq.floquet_batch_destroy(b)
        print(f"ncu case scan: N = {[p.n for p in plans]}, L = {[p.info.L for p in plans]}, "
              f"status {[p.check_status() for p in plans]}")
        return
    if case == "split":
        m = fi.config_goe4096()
        plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=m.drive.f_ac, steps=m.steps,
                             precision=fq.FQ_BF16X3)
        x0 = torch.zeros((4096, 4096), dtype=torch.complex128, device="cuda")
        x0.diagonal().fill_(1.0)
        ws = fq.workspace(plan.workspace_size(4096))
        for _ in range(2):
            fq.floquet_propagate(plan.handle, x0, x0, 4096, 0, 1, ws)
        torch.cuda.synchronize()
        print(f"ncu case split: status {plan.check_status()}")
        return
    d = fi.config_dimer(nb=NB, steps=STEPS)
    n = d.n
    kernel = {"resident": fq.FQ_KERNEL_RESIDENT, "stream": fq.FQ_KERNEL_STREAM, "tile": fq.FQ_KERNEL_TILED,
              "dfl": fq.FQ_KERNEL_TILED, "band": fq.FQ_KERNEL_BAND}[case]
    precision = {"tile": fq.FQ_FP64, "dfl": fq.FQ_DF32, "band": fq.FQ_OZAKI}.get(case, fq.FQ_FP32)
    plan = fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=d.drive.omega, f_ac=d.drive.f_ac,
                           steps=d.steps, precision=precision, kernel=kernel)
    nc, m_end = {"resident": (152, 20), "band": (4096, 3)}.get(case, (2048, 1))
    x0 = torch.zeros((nc, n), dtype=torch.complex128, device="cuda")
    x0[torch.arange(nc), torch.arange(nc) * (n // nc)] = 1.0
    ws = fq.workspace(plan.workspace_size(nc))
    x = x0 if case == "band" else torch.empty_like(x0)  # (in place: the band case's states are larger)
    for _ in range(2):
        fq.floquet_propagate(plan.handle, x0, x, nc, 0, m_end, ws)
    torch.cuda.synchronize()
    print(f"ncu case {case}: {nc} states, steps 0..{m_end - 1}, status {plan.check_status()}")


def measured_peaks():
    """The driver-written measured peaks (HBM copy, cuBLAS bf16 burst and sustained), else the
    earlier fallback measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return {"hbm_gbs": m["hbm_gbs"], "bf16": m["bf16_tflops"], "bf16_sustained": m["bf16_tflops_sustained"],
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_drive_amplitude(base: float, rank: int) -> float:
    """Weak scaling: rank r builds the U_T of its own drive amplitude eps1 = base + 0.01 r (an
    independent problem of identical cost); rank 0 runs exactly the benchmark workload."""
    return base + 0.01 * rank


def job_throughput(local_seconds: float, steps: int, dist=None, device=None) -> tuple[float, float]:
    """Whole-job U_T/s: every rank did `steps` builds; the job took the slowest rank's time
    (max over ranks, no data-path collective).  Returns (value, max_seconds)."""
    world = 1
    total = local_seconds
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return world * steps / total, total


# ---------------------------------------------------------------------- oracle timing
def _oracle_worker_init():
    # one thread per process: the oracle's tridiagonal products are elementwise numpy
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"


def _oracle_ready(_):
    import numpy  # noqa: F401
    import oracle  # noqa: F401
    return os.getpid()


def _oracle_block(job):
    """One block of basis states through `steps` steps of the oracle's chain (worker process)."""
    import numpy as np
    import oracle as o
    d, plan, idx, steps = job
    x0 = np.zeros((d.n, len(idx)), complex)
    x0[idx, np.arange(len(idx))] = 1.0
    return x0, o.propagate_tridiag(d.h0_diag, d.h0_off, d.h1_diag, plan, x0, 0, steps)


def oracle_sample(cols_per_core=6, steps=100, d=None, cores=None):
    """FP64 oracle on cols_per_core basis states per host core over `steps` of the workload's
    chain (default: the M = 2000 dimer), one spawned process per core; returns (U_T builds per
    second scaled to the full workload, seconds, description, cores, (x0, x, steps))."""
    import multiprocessing as mp
    import numpy as np
    import floquet_inputs as fi
    import oracle as o
    if d is None:
        d = fi.config_dimer(nb=NB, steps=STEPS)
    cores = cores or os.cpu_count() or 1
    cols = cols_per_core * cores
    plan = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    idx = np.linspace(0, d.n - 1, cols).astype(int)
    blocks = np.array_split(idx, cores)
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_ready, range(cores))  # workers started and imported before timing
        t0 = time.perf_counter()
        outs = pool.map(_oracle_block, [(d, plan, b, steps) for b in blocks])
        dt = time.perf_counter() - t0
    x0 = np.concatenate([a for a, _ in outs], axis=1)
    x = np.concatenate([b for _, b in outs], axis=1)
    frac = (cols / d.n) * (steps / d.steps)
    desc = (f"{cols} of {d.n} basis states over {steps} of {d.steps} steps (FP64 numpy oracle, {cores} processes "
            f"x 1 thread)")
    return frac / dt, dt, desc, cores, (x0, x, steps)


def host_info():
    """Host cores and CPU model (the oracle baseline runs on them)."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    model = arm_parts.get(model.lower(), model)
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import floquet_inputs  # noqa: F401
    for _ in range(args.warmup):
        oracle_sample(cols_per_core=1, steps=20)
    vals, secs = [], 0.0
    desc, cores = "", 1
    for _ in range(args.steps):
        v, dt, desc, cores, _ = oracle_sample()
        vals.append(v)
        secs += dt
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": "U_T builds/sec (dim 10001 Bose-Hubbard dimer, M=2000, FP64-level)",
            "value": value, "unit": "U_T/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "bose-hubbard dimer nb=10000 (dim 10001), M=2000, L=39",
                       "kernel": "FP64 numpy oracle (host cores)"},
            "cpu_baseline": {"value": value, "unit": "U_T/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "U_T/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- our arm
# The dimer kernels the bench times, with how one launch's work is counted for the roofline; the
# unit is the element-term (one entry of one state through one Chebyshev product).
DIMER_PATHS = {
    # FP32 resident chain (one launch per U_T): 26 flop per element-term against the FP32 FMA peak
    "fp32": {"precision": "FQ_FP32", "kernel": "FQ_KERNEL_RESIDENT", "dtype": "f32", "level": "FP32",
             "kernel_name": "k_tri_resident<256, 40>", "unit": "TFLOP/s", "per_unit": FLOPS_PER_ELEMENT_TERM,
             "launches_per_step": 2,
             "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived from unit counts and clocks)"},
    # double-float tiled chain (FP64-level, one launch per step): 4 double-float complex FMAs per
    # element-term, each 15 packed FP32x2 operations (30 FP32 lane operations), against the FP32
    # lane-operation peak
    # band kernel (FP64-level, FQ_OZAKI): per step the band matrix of the step's polynomial times
    # every state on the tensor cores in FP64 emulation; 26 flop per element-term of the method
    # (as the FP32 line counts it) against the measured sustained bf16 peak, with the issued
    # slice-product rate beside it
    "ozaki": {"precision": "FQ_OZAKI", "kernel": "FQ_KERNEL_BAND", "dtype": "ozaki (bf16 slices, fp32 sums)",
              "level": "FP64", "kernel_name": "k_oz_band", "unit": "TFLOP/s", "per_unit": FLOPS_PER_ELEMENT_TERM,
              # per U_T build: the product and the fixup pass of every step, plus the gauge tables, the
              # load, the first step's row maxima, slices and band, and the store (10001 states: the
              # product forms the next band itself)
              "launches_per_step": 2 * STEPS + 6, "tensor": True,
              "peak_note": "measured sustained cuBLAS bf16 (MEASURED_PEAKS.json)"},
    "df32": {"precision": "FQ_DF32", "kernel": "FQ_KERNEL_TILED", "dtype": "df32 (FP32 pairs, FP64 states)",
             "level": "FP64", "kernel_name": "k_tri_tile_dfl", "unit": "Tops/s",
             "per_unit": DFL_LANE_OPS_PER_ELEMENT_TERM, "launches_per_step": STEPS + 3,
             "peak_note": "FP32 lane operations: 152 SMs x 128 lanes x 2070 MHz (derived from unit counts and clocks)"},
}


# DRAM bytes of one k_oz_band launch (one step's banded product) from the ncu capture of
# `python bench.py --ncu-case band` (4096 states; profiles/k_oz_band_dimer10001.md), scaled to a
# launch by states: the state slices read and the next step's slices written grow with the states
# (a step that is not the last: no double-float states written).
BAND_NCU = {"read": 1140.6e6, "write": 989.4e6, "states": 4096}


def band_window(L):
    """K width of the band kernel's tiles: 64 operator rows plus L rounded up to a multiple of 8
    (at most 48) on each side."""
    return 64 + 2 * min(48, -(-L // 8) * 8)


def band_issued_flops(n, nc, L):
    """BF16 MMA flops the band kernel issues per step: tiles of 128 states x 64 operator rows, a
    K window of band_window(L) columns, 21 slice pairs of two N = 128 MMAs."""
    tiles = -(-nc // 128) * -(-n // 64)
    return tiles * 21 * 2 * 2.0 * 128 * 128 * band_window(L)


def dimer_roofline(path, n, steps, L, seconds_per_launch, per_launch_units):
    """Roofline of the dominant dimer kernel: algorithmic work of one launch / its CUDA-event time."""
    work = path["per_unit"] * per_launch_units
    achieved = work / seconds_per_launch / 1e12
    if path.get("tensor"):
        peak = measured_peaks()["bf16_sustained"]
        issued = band_issued_flops(n, n, L) * per_launch_units / (float(n) * n * L) / seconds_per_launch / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "kernel": path["kernel_name"], "work_per_unit": path["per_unit"],
                "units_per_launch": per_launch_units, "issued_tflops": issued, "issued_frac": issued / peak,
                "peak_note": path["peak_note"] + " (" + measured_peaks()["source"] + ")",
                "work_note": "achieved counts the method's 26 flop per element-term (useful work, as the FP32 "
                             "line); issued counts the BF16 slice products the emulation runs"}
    if path["unit"] == "TFLOP/s":
        peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    else:
        peak = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": path["unit"], "frac": achieved / peak,
            "kernel": path["kernel_name"], "work_per_unit": path["per_unit"], "units_per_launch": per_launch_units,
            "peak_note": path["peak_note"]}


def measured_fp32_rate(fq, torch, stream):
    """The GPU's FP32 multiply-add rate, measured live by the library's probe (4 CTAs of 256 threads
    per SM, independent chains): CUDA events around 5 launches after 3 warm-ups, packed (FFMA2) and
    scalar (FFMA), in TFLOP/s."""
    out = torch.empty(4 * SM_COUNT * 256, dtype=torch.float32, device="cuda")
    rates = {}
    for packed, key in ((True, "ffma2"), (False, "ffma")):
        for _ in range(3):
            fq.floquet_probe_fp32(packed, 16384, out, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = sum(fq.floquet_probe_fp32(packed, 16384, out, stream) for _ in range(5))
        e1.record(stream)
        e1.synchronize()
        rates[key] = flops / (e0.elapsed_time(e1) / 1e3) / 1e12
    return rates


def with_measured_fp32(roof, rates):
    """The FP32 roofline entry with the live-measured FP32 rate beside the derived peak."""
    roof = dict(roof)
    roof["peak_measured"] = rates["ffma2"]
    roof["peak_measured_scalar"] = rates["ffma"]
    roof["frac_of_measured"] = roof["achieved"] / rates["ffma2"]
    roof["peak_measured_note"] = ("FP32 multiply-add rate of floquet_probe_fp32 (packed FFMA2; scalar FFMA "
                                  "beside it), CUDA events over 5 launches in this run")
    return roof


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import floquet_inputs as fi
    import paper_1508_07621_gb300 as fq
    from paper_1508_07621_gb300 import shard

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    paper = args.workload == "dimer-paper"
    prec = args.precision or "ozaki"
    if prec not in DIMER_PATHS:
        raise SystemExit(f"--precision for the dimer: one of {sorted(DIMER_PATHS)}")
    path = DIMER_PATHS[prec]
    d = fi.config_dimer_paper(nb=NB, steps=8000) if paper else fi.config_dimer(nb=NB, steps=STEPS)
    sharded = world > 1 and args.shard == "columns"
    # replicas: rank r builds the U_T of its own drive amplitude; columns: all ranks share one U_T
    f_ac = d.drive.f_ac if sharded else rank_drive_amplitude(d.drive.f_ac, rank)
    f_dc = d.drive.f_dc
    n = d.n
    stream = torch.cuda.current_stream()

    def make_plan(p):
        return fq.Plan.tridiag(d.h0_diag, d.h0_off, d.h1_diag, omega=d.drive.omega, f_ac=f_ac, f_dc=f_dc,
                               steps=d.steps, precision=getattr(fq, p["precision"]), kernel=getattr(fq, p["kernel"]))

    def timed_build(p, warmup, steps):
        """Warm-up, then `steps` CUDA-event-timed U_T builds of path p; returns the plan, the last
        U_T (row-major, or column-major when sharded), per-step seconds, total seconds, clocks."""
        plan = make_plan(p)
        if sharded:
            buf = shard.gather_buffer(n, world)
            ws = shard.columns_workspace(plan, world)
            out = {}

            def step():
                out["U"] = shard.build_ut_sharded(plan, dist, buf, ws, stream)
        else:
            ws = fq.workspace(plan.workspace_size())
            U = torch.empty((n, n), dtype=torch.complex128, device="cuda")
            out = {"U": U}

            def step():
                fq.floquet_build_UT(plan.handle, U, ws, stream)
        for _ in range(max(warmup, 0)):
            step()
        torch.cuda.synchronize()
        if plan.check_status() != fq.FQ_OK:
            raise RuntimeError("device bound check fired during warm-up")
        # CUDA events around every launch of the step kernel, on its stream, over the timed region
        fq.floquet_kernel_timing(plan.handle, True)
        per_step, total, clk = timed_loop(step, steps, stream, world, dist)
        ktime = fq.floquet_kernel_time(plan.handle)
        fq.floquet_kernel_timing(plan.handle, False)
        return plan, out["U"], per_step, total, clk, ktime

    plan, U, per_step, total, clk, ktime = timed_build(path, args.warmup, args.steps)
    value, total = job_throughput(total, args.steps, dist if world > 1 else None, "cuda")
    if sharded:
        value /= world  # every rank took part in the same U_T builds
    L = plan.info.L
    status_ok = plan.check_status() == fq.FQ_OK
    # accuracy of the timed result: unitarity defect over 64 sampled columns (FP64, on the GPU);
    # the sharded result is column-major, whose row defect is that of U_T's columns
    sample_cols = torch.arange(0, n, n // 64, dtype=torch.int32, device="cuda")[:64]
    Urm = U.mT.contiguous() if sharded else U
    defect_max, defect_fro = fq.api.unitarity_defect(Urm, sample_cols)
    del Urm

    # end to end through the C ABI with host buffers: plan from host arrays (H2D inside the
    # call), build, and the D2H copy of U_T into pinned host memory, every step
    host_u = torch.empty((n, n), dtype=torch.complex128, pin_memory=True)
    e2e_times = []
    h2d = 8 * (n + n + (n - 1)) + 8 * (n - 1) + 3 * 8 * d.steps
    # caller-owned device buffers, allocated once as a user would: the output (U above, or the
    # gather buffer) and the workspace
    if sharded:
        ebuf, ews = shard.gather_buffer(n, world), shard.columns_workspace(plan, world)
    else:
        ews = fq.workspace(plan.workspace_size())
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        p2 = make_plan(path)
        if sharded:
            Ue = shard.build_ut_sharded(p2, dist, ebuf, ews, stream)
        else:
            Ue = U
            fq.floquet_build_UT(p2.handle, Ue, ews, stream)
        host_u.copy_(Ue, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        p2.close()
        del Ue
    e2e_local = statistics.median(e2e_times) if e2e_times else float("nan")
    e2e_value, _ = job_throughput(e2e_local, 1, dist if world > 1 else None, "cuda")
    if sharded:
        e2e_value /= world

    # the FP32 resident kernel alongside an FP64-level headline (same workload, its own timing)
    fp32 = None
    if prec != "fp32" and not args.no_fp32_extra:
        p32, _, ps32, tot32, clk32, kt32 = timed_build(DIMER_PATHS["fp32"], min(args.warmup, 3), args.fp32_steps)
        v32, tot32 = job_throughput(tot32, args.fp32_steps, dist if world > 1 else None, "cuda")
        if sharded:
            v32 /= world
        avg32 = kt32[1] / 1000.0 / kt32[0] if kt32[0] else statistics.mean(ps32)
        fp32 = {"value": v32, "unit": "U_T/s", "ms_per_step": 1000.0 * tot32 / args.fp32_steps,
                "steps": args.fp32_steps, "dtype": "f32", "per_step_s": ps32, "clocks": clk32,
                "roofline": with_measured_fp32(
                    dict(dimer_roofline(DIMER_PATHS["fp32"], n, d.steps, L, avg32,
                                        float(n) * n * d.steps * L / (world if sharded else 1)),
                         traffic=resident_traffic(n, d.steps, n / (world if sharded else 1)),
                         traffic_note=RES_TRAFFIC_NOTE), measured_fp32_rate(fq, torch, stream))}
        p32.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    avg = statistics.mean(per_step)
    # the step kernel's mean launch duration from its own events (else the build time per launch)
    klaunches, kms, kname = ktime
    if prec == "fp32":  # one launch per U_T: the whole chain
        kavg = kms / 1000.0 / klaunches if klaunches else avg
        roofline = dimer_roofline(path, n, d.steps, L, kavg, float(n) * n * d.steps * L / (world if sharded else 1))
        roofline["traffic"] = resident_traffic(n, d.steps, n / (world if sharded else 1))
        roofline["traffic_note"] = RES_TRAFFIC_NOTE
        roofline = with_measured_fp32(roofline, measured_fp32_rate(fq, torch, stream))
    else:  # one launch per step: units of one launch over the launch's mean duration
        per_launch = float(n) * n * L / (world if sharded else 1)
        kavg = kms / 1000.0 / klaunches if klaunches else avg / d.steps
        roofline = dimer_roofline(path, n, d.steps, L, kavg, per_launch)
        roofline["traffic"] = None
        roofline["traffic_note"] = "see profiles/ for the kernel's DRAM bytes per launch"
        if prec == "ozaki" and BAND_NCU["read"] is not None:
            roofline["traffic"] = (BAND_NCU["read"] + BAND_NCU["write"]) * (n / (world if sharded else 1)) / \
                BAND_NCU["states"]
            roofline["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of k_oz_band from one ncu capture "
                                        "of --ncu-case band (4096 states), scaled to a launch by states")
    roofline["launch_seconds"] = kavg
    roofline["launch_seconds_note"] = (
        f"mean of {klaunches} CUDA-event-timed launches of {kname} on its stream over the timed region "
        "(floquet_kernel_timing); the U_T time also holds the step's other launches (profiles' launch list)"
        if klaunches else "mean U_T time / launches per U_T (no kernel events recorded)")
    cpu = None
    accuracy = {"unitarity_defect_max": defect_max, "unitarity_defect_fro": defect_fro,
                "defect_columns": int(sample_cols.numel())}
    if not args.no_cpu_baseline and world == 1:
        v, dt, desc, cores, (x0s, xs, nst) = oracle_sample(d=d)
        cpu = {"value": v, "unit": "U_T/s", "cores": cores, "kind": "oracle", "sample": desc}
        # the same states through the same steps on the library: max-abs difference to the oracle
        rows = torch.from_numpy(np.ascontiguousarray(x0s.T)).to("cuda")
        got = plan.propagate(rows, 0, nst).cpu().numpy().T
        accuracy["sample_max_err_vs_oracle"] = float(np.max(np.abs(got - xs)))
        accuracy["sample"] = desc
    tag = ", paper parameters" if paper else ""
    parallelism = (f"columns: {world} ranks share each U_T (column blocks + one all-gather)" if sharded
                   else f"replicas: {world} independent drive amplitudes" if world > 1 else "1 GPU")
    line = {"metric": f"U_T builds/sec (dim {n} Bose-Hubbard dimer{tag}, M={d.steps}, {path['level']}-level)",
            "value": value, "unit": "U_T/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
            "dtype": path["dtype"], "data": "synthetic",
            "config": {"workload": f"bose-hubbard dimer{tag} nb={n - 1} (dim {n}), M={d.steps}, L={L}",
                       "kernel": f"{path['level']}-level arithmetic on {path['kernel_name']}",
                       "dim": n, "steps_per_period": d.steps, "chebyshev_L": L, "R": plan.info.R,
                       "delta_e": plan.info.delta_e,
                       "l2": "working set larger than L2 (U_T 1.6 GB; per-step operator coefficients)",
                       "parallelism": parallelism},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "U_T/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * n * n},
            "gpu_launches": path["launches_per_step"] * args.steps, "clocks": clk, "device_status_ok": status_ok,
            "accuracy": accuracy, "median_step_s": statistics.median(per_step), "per_step_s": per_step,
            "host": host_info()}
    if fp32 is not None:
        line["fp32"] = fp32
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------- dense and gradient workloads
PREC_NAMES = {"x3": "FQ_BF16X3", "x6": "FQ_BF16X6", "ozaki": "FQ_OZAKI", "fp64": "FQ_FP64"}
SLICE_PRODUCTS = {"x3": 3, "x6": 6, "ozaki": 21, "fp64": 1}


def timed_loop(fn, steps, stream, world, dist):
    """CUDA-event timing of `steps` calls of fn on `stream`, barrier + synchronize on both sides;
    returns (per-call seconds, total seconds, clock record)."""
    import torch
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.5)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(steps):
        fn()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    return [ev[k].elapsed_time(ev[k + 1]) / 1000.0 for k in range(steps)], ev[0].elapsed_time(ev[-1]) / 1000.0, clk


def dense_oracle_sample(m, states=64, steps=4, cheb_terms=0):
    """FP64 oracle (numpy, BLAS on every host core) on `states` basis states over the first `steps`
    steps of the dense workload; returns (U_T/s scaled to the full build, seconds, description,
    (idx, x, steps)).  cheb_terms > 0 fixes L (its weights from the oracle's own Bessel routine)."""
    import dataclasses
    import numpy as np
    import oracle as o
    plan = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    if cheb_terms:
        plan = dataclasses.replace(plan, L=cheb_terms, coeffs=o.bessel_coefficients(plan.R, cheb_terms))
    idx = np.linspace(0, m.n - 1, states).astype(int)
    x0 = np.zeros((m.n, states), complex)
    x0[idx, np.arange(states)] = 1.0
    t0 = time.perf_counter()
    x = o.propagate_dense(m.h0, m.h1, plan, x0, 0, steps)
    dt = time.perf_counter() - t0
    frac = (states / m.n) * (steps / m.steps)
    desc = f"{states} of {m.n} basis states over {steps} of {m.steps} steps (FP64 numpy oracle, BLAS threads)"
    if cheb_terms:
        desc += f", L = {cheb_terms}, 4th-order operator (the L products per step dominate)"
    return frac / dt, dt, desc, (idx, x, steps)


def adjoint_oracle_sample(a, steps=2):
    """FP64 oracle gradient of the sub-problem made of the first `steps` steps (same N, same step
    length); returns (gradients/s scaled to M steps, seconds, description, (loss, g, f, T))."""
    import oracle as o
    M = len(a.f)
    fm = a.f[:steps]
    T = a.period * steps / M
    plan = o.plan_piecewise(a.h0, a.h1, T, fm)
    t0 = time.perf_counter()
    loss, g = o.grad_piecewise(a.h0, a.h1, a.target, plan, fm)
    dt = time.perf_counter() - t0
    desc = (f"oracle gradient of the first {steps} of {M} steps at N = {a.h0.shape[0]} (FP64 numpy, BLAS "
            f"threads), scaled by {M}/{steps}")
    return (steps / M) / dt, dt, desc, (loss, g, fm, T)


def run_dense(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import floquet_inputs as fi
    import paper_1508_07621_gb300 as fq

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    paper = args.workload == "paper-table1"
    prec = args.precision or ("ozaki" if paper else "x3")
    if prec == "fp64":
        raise SystemExit("N = 4096 in plain FP64 takes many minutes per U_T; use x3, x6 or ozaki")
    m = fi.config_goe_paper(args.n) if paper else fi.config_goe4096()
    order, terms = (6, 50) if paper else (0, 0)
    f_ac = rank_drive_amplitude(m.drive.f_ac, rank)
    n = m.n
    precision = getattr(fq, PREC_NAMES[prec])
    stream = torch.cuda.current_stream()
    plan = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=f_ac, steps=m.steps, precision=precision,
                         magnus_order=order, cheb_terms=terms)
    ws = fq.workspace(plan.workspace_size())
    tile = plan.autotune(ws) if prec != "ozaki" else 0
    L = plan.info.L
    U = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    for _ in range(max(args.warmup, 0)):
        fq.floquet_build_UT(plan.handle, U, ws, stream)
    torch.cuda.synchronize()
    if plan.check_status() != fq.FQ_OK:
        raise RuntimeError("device check fired during warm-up")
    per_step, total, clk = timed_loop(lambda: fq.floquet_build_UT(plan.handle, U, ws, stream), args.steps, stream,
                                      world, dist)
    value, total = job_throughput(total, args.steps, dist if world > 1 else None, "cuda")
    status_ok = plan.check_status() == fq.FQ_OK
    sample_cols = torch.arange(0, n, n // 64, dtype=torch.int32, device="cuda")[:64]
    defect_max, defect_fro = fq.api.unitarity_defect(U, sample_cols)
    # end to end: plan from host arrays (H0, H1 uploaded inside the call), build, U_T to pinned host
    host_u = torch.empty((n, n), dtype=torch.complex128, pin_memory=True)
    e2e_times = []
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = fq.Plan.dense(m.h0, m.h1, omega=m.drive.omega, f_ac=f_ac, steps=m.steps, precision=precision,
                           tile_n=tile, magnus_order=order, cheb_terms=terms)
        fq.floquet_build_UT(p2.handle, U, ws, stream)
        host_u.copy_(U, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        p2.close()
    e2e_value = world / statistics.median(e2e_times) if e2e_times else None
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    useful = 8.0 * n ** 3 * L * m.steps
    issued = useful * SLICE_PRODUCTS[prec]
    avg = statistics.mean(per_step)
    achieved = useful / avg / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16_sustained"], "traffic": None,
                "kernel": "k_oz_term" if prec == "ozaki" else "k_split_persist",
                "issued_tflops": issued / avg / 1e12, "issued_frac": issued / avg / 1e12 / peaks["bf16_sustained"],
                "note": (f"achieved: useful 8 N^3 flop per term x M L terms per build; issued: the "
                         f"{SLICE_PRODUCTS[prec]} BF16 slice products each term runs; both over the build's "
                         "CUDA-event time (the operator and slicing kernels, a few percent, included); peak: "
                         f"{peaks['source']} sustained cuBLAS bf16 (a build is seconds of back-to-back GEMMs)")}
    accuracy = {"unitarity_defect_max": defect_max, "unitarity_defect_fro": defect_fro,
                "defect_columns": int(sample_cols.numel())}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, desc, (idx, xs, nst) = dense_oracle_sample(m, steps=2 if paper else 4, cheb_terms=terms)
        cpu = {"value": v, "unit": "U_T/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}
        if not paper:  # (the paper's run is 6th order; the oracle sample times the 4th-order chain)
            rows = torch.zeros((len(idx), n), dtype=torch.complex128, device="cuda")
            rows[torch.arange(len(idx)), torch.as_tensor(idx, device="cuda")] = 1.0
            got = plan.propagate(rows, 0, nst).cpu().numpy().T
            accuracy["sample_max_err_vs_oracle"] = float(np.max(np.abs(got - xs)))
            accuracy["sample"] = desc
    launches = 2 + m.steps * (1 + (2 * L if prec == "ozaki" else L))
    if paper:
        metric = (f"U_T builds/sec (the paper's Table 1 timing run: GOE N={n} with unit-variance entries, "
                  f"f = cos(pi t), M={m.steps}, L={L}, 6th-order Magnus)")
        vs = value * PAPER_TABLE1_CHEB_S[n]
        workload = (f"paper Table 1: GOE N={n} (seeds 3, 4, unit-variance entries), f=cos(pi t), T=2, M={m.steps}, "
                    f"L={L} fixed, 6th-order Magnus, {PREC_NAMES[prec]}")
    else:
        metric, vs = f"U_T builds/sec (dense GOE N={n}, M={m.steps})", None
        workload = f"dense GOE N={n} (seeds 3, 4), A=2, omega=2, M={m.steps}, L={L}, {PREC_NAMES[prec]}"
    line = {"metric": metric, "value": value, "unit": "U_T/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": vs,
            "dtype": "bf16 slices, f64 states" if prec == "ozaki" else "bf16 slices, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": workload,
                       "n": n, "steps_per_period": m.steps, "chebyshev_L": L, "R": plan.info.R, "tile_n": tile,
                       "l2": "working set larger than L2 (operand slices and states, > 1 GB)",
                       "parallelism": f"weak: {world} independent drive amplitudes"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "U_T/s", "h2d_bytes_per_step": 16 * n * n + 24 * m.steps,
                    "d2h_bytes_per_step": 16 * n * n},
            "gpu_launches": launches * args.steps, "clocks": clk, "device_status_ok": status_ok,
            "accuracy": accuracy, "median_step_s": statistics.median(per_step), "per_step_s": per_step,
            "host": host_info()}
    # the quasienergies (Eq. 5) from the timed U_T by host FP64 LAPACK zgeev, outside the timed
    # region (the paper's Table 1 lists it separately)
    t0 = time.perf_counter()
    eps, _ = fq.floquet_states(U, m.drive.period)
    line["quasienergies"] = {"host_zgeev_s": time.perf_counter() - t0, "count": int(len(eps)),
                             "cores": os.cpu_count()}
    if paper:
        line["vs_baseline_note"] = (f"value x {PAPER_TABLE1_CHEB_S[n]} s: the paper's Chebyshev-iteration time for one "
                                    "U_T of this run on one 16-core Xeon node in FP64 (Table 1); context, not a "
                                    "target (another machine)")
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


BATCH_STEPS = 256


def batch_mma_flops(insts, Ls, tiles, prec, scan):
    """Tensor-core work the scan issues, padding included: per term, 128-row state blocks x the
    output rows of whole tiles x K rounded up to the stage depth, times the slice products.  The
    persistent scan runs one tile width for every instance (the one the plans' widths favour,
    weighted by N^3 L); the lane graph runs each plan's own."""
    def ceil(x, b):
        return -(-x // b) * b
    if prec not in ("x3", "x6"):
        return None
    if scan:
        w = {64: 0.0, 128: 0.0}
        for s, L, t in zip(insts, Ls, tiles):
            w[128 if t == 128 else 64] += float(s.n) ** 3 * L
        tiles = [128 if w[128] >= w[64] else 64] * len(insts)
    tot = 0.0
    for s, L, t in zip(insts, Ls, tiles):
        bke = 32 if (prec == "x6" or t == 128) else 64
        tot += 8.0 * ceil(s.n, 128) * ceil(s.n, 128) * ceil(s.n, bke) * L * BATCH_STEPS
    return tot * SLICE_PRODUCTS[prec]


def batch_flops(insts, Ls):
    """Useful flop of one scan: 8 N^3 per Chebyshev term (a complex N x N product as real
    products), L terms per step, M steps per instance."""
    return sum(8.0 * s.n ** 3 * L * BATCH_STEPS for s, L in zip(insts, Ls))


def batch_oracle_sample(insts, states=None, steps=16):
    """FP64 oracle on `states` basis states over `steps` steps of the scan's first instance,
    scaled to the whole scan by each instance's share of N^3 L (the oracle's products are BLAS
    GEMMs, so its time follows the flop count); returns (instances/s, seconds, description).
    L_i for the scaling comes from the oracle's truncation rule at R_i = h_i (2 + 2 A_i): the
    GOE matrices of the scan have spectral radius 2, so |H0 + f H1| <= 2 + 2 |A|."""
    import math
    import oracle as o
    import floquet_inputs as fi
    m0 = fi.scan_model(insts[0], BATCH_STEPS)
    # the whole identity block of instance 0 by default: narrower blocks run the oracle's BLAS
    # products below their speed and overstate its time
    v0, dt, desc0, _ = dense_oracle_sample(m0, states=states or m0.n, steps=steps)
    est = [o.chebyshev_order(2 * math.pi / s.omega / BATCH_STEPS * (2 + 2 * s.amplitude)) for s in insts]
    scale = sum((s.n / m0.n) ** 3 * (est[i] / est[0]) for i, s in enumerate(insts))
    t_scan = scale / v0  # seconds for the whole scan: v0 is instance 0's U_T/s
    desc = (f"{desc0} of instance 0 (N = {m0.n}), scaled to the {len(insts)}-instance scan by sum (N_i / N_0)^3 "
            f"(L_i / L_0) with L_i from R_i = h_i (2 + 2 A_i)")
    return len(insts) / t_scan, dt, desc


def run_batch(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import floquet_inputs as fi
    import paper_1508_07621_gb300 as fq

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = args.precision or "x3"
    if prec == "fp64":
        raise SystemExit("the scan's N = 2048 instances take minutes each in plain FP64; use x3, x6 or ozaki")
    precision = getattr(fq, PREC_NAMES[prec])
    insts = fi.batch_scan()
    # weak scaling: rank r scans amplitudes shifted by 0.01 r (independent problems of the same cost)
    models = [(fi.goe(s.n, s.seed_h0), fi.goe(s.n, s.seed_h1), s.omega, rank_drive_amplitude(s.amplitude, rank))
              for s in insts]

    def make_plans(tiles=None):
        return [fq.Plan.dense(h0, h1, omega=om, f_ac=amp, steps=BATCH_STEPS, precision=precision,
                              tile_n=tiles[i] if tiles else 0)
                for i, (h0, h1, om, amp) in enumerate(models)]

    stream = torch.cuda.current_stream()
    plans = make_plans()
    ws1 = fq.workspace(max(p.workspace_size() for p in plans))
    tiles = [p.autotune(ws1) if prec != "ozaki" else 0 for p in plans]
    del ws1
    Ls = [p.info.L for p in plans]
    outs = [torch.empty((p.n, p.n), dtype=torch.complex128, device="cuda") for p in plans]
    handles = [p.handle for p in plans]
    ws = fq.workspace(fq.floquet_batch_workspace_size(handles))
    # the persistent scan takes split-precision plans with L <= 32; anything else runs on 8 lanes
    scan = args.lanes == 0 and prec in ("x3", "x6") and max(Ls) <= 32
    lanes = 0 if scan else (args.lanes or 8)
    graph = fq.floquet_batch_create(handles, outs, ws, lanes)
    try:
        for _ in range(max(args.warmup, 0)):
            fq.floquet_batch_launch(graph, stream)
        torch.cuda.synchronize()
        if any(p.check_status() != fq.FQ_OK for p in plans):
            raise RuntimeError("device check fired during warm-up")
        per_step, total, clk = timed_loop(lambda: fq.floquet_batch_launch(graph, stream), args.steps, stream,
                                          world, dist)
    finally:
        fq.floquet_batch_destroy(graph)
    status_ok = all(p.check_status() == fq.FQ_OK for p in plans)
    value, total = job_throughput(total, args.steps, dist if world > 1 else None, "cuda")
    value *= len(plans)  # instances/s: each launch builds every instance's U_T
    defect = max(fq.api.unitarity_defect(u, torch.arange(0, u.shape[0], max(1, u.shape[0] // 16),
                                                         dtype=torch.int32, device="cuda")[:16])[0]
                 for u in outs)
    # end to end: every plan from host arrays, the graph, one launch, every U_T to pinned host
    host = [torch.empty(tuple(u.shape), dtype=torch.complex128, pin_memory=True) for u in outs]
    e2e_times = []
    for _ in range(min(args.e2e_steps, 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = make_plans(tiles)
        g2 = fq.floquet_batch_create([p.handle for p in p2], outs, ws, lanes)
        fq.floquet_batch_launch(g2, stream)
        for h, u in zip(host, outs):
            h.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        fq.floquet_batch_destroy(g2)
        for p in p2:
            p.close()
    e2e_value = world * len(plans) / statistics.median(e2e_times) if e2e_times else None
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    useful = batch_flops(insts, Ls)
    issued = useful * SLICE_PRODUCTS[prec]
    padded = batch_mma_flops(insts, Ls, tiles, prec, scan)
    avg = statistics.mean(per_step)
    achieved = useful / avg / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16_sustained"], "traffic": None,
                "kernel": "k_split_scan" if scan else ("k_oz_term" if prec == "ozaki" else "k_split_persist"),
                "issued_tflops": issued / avg / 1e12, "issued_frac": issued / avg / 1e12 / peaks["bf16_sustained"],
                "issued_with_padding_frac": (padded / avg / 1e12 / peaks["bf16_sustained"]) if padded else None,
                "note": (f"achieved: useful 8 N_i^3 L_i M flop summed over the {len(plans)} instances; issued: "
                         f"x {SLICE_PRODUCTS[prec]} BF16 slice products; issued_with_padding: the MMAs as run, "
                         f"on whole 128-state blocks, whole output tiles and K rounded up to the stage depth; all "
                         f"over one graph launch's CUDA-event time; peak: {peaks['source']} sustained cuBLAS bf16")}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, desc = batch_oracle_sample(insts)
        cpu = {"value": v, "unit": "instances/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}
    # kernels per graph launch: the one persistent kernel, or per instance its init, store and per
    # step the Omega~ slices and L terms (2 L with the FP64 emulation's fix-ups)
    launches = 1 if scan else sum(2 + BATCH_STEPS * (1 + (2 * L if prec == "ozaki" else L)) for L in Ls)
    ns = [s.n for s in insts]
    line = {"metric": f"instances/sec ({len(plans)}-instance dense GOE scan, N ~ U{{256..2048}}, M={BATCH_STEPS}, "
                      "one CUDA graph)",
            "value": value, "unit": "instances/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 slices, f64 states" if prec == "ozaki" else "bf16 slices, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": (f"batched scan: {len(plans)} GOE instances (seeds 1000 + 2i, 1001 + 2i), "
                                    f"N in [{min(ns)}, {max(ns)}], omega ~ U[0.5, 4], A ~ U[0.5, 3], M={BATCH_STEPS}, "
                                    f"{PREC_NAMES[prec]}, "
                                    + ("one persistent launch over work units" if scan else f"{lanes} graph lanes")),
                       "instances": len(plans), "lanes": lanes, "L_range": [min(Ls), max(Ls)],
                       "tiles": tiles,
                       "l2": "working set larger than L2 (operand slices and states of 48 instances, > 1 GB)",
                       "parallelism": f"weak: {world} independent scans"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "instances/s",
                    "h2d_bytes_per_step": sum(16 * n * n + 24 * BATCH_STEPS for n in ns),
                    "d2h_bytes_per_step": sum(16 * n * n for n in ns)},
            "gpu_launches": launches * args.steps, "clocks": clk, "device_status_ok": status_ok,
            "accuracy": {"unitarity_defect_max": defect, "defect_columns_per_instance": 16},
            "median_step_s": statistics.median(per_step), "per_step_s": per_step, "host": host_info()}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_adjoint(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import floquet_inputs as fi
    import paper_1508_07621_gb300 as fq

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = args.precision or "x3"
    a = fi.config_adjoint()
    n, M = a.h0.shape[0], len(a.f)
    fm = a.f + 0.01 * rank  # rank r: its own initial amplitudes (an independent problem)
    precision = getattr(fq, PREC_NAMES[prec])
    stream = torch.cuda.current_stream()
    tile = 64 if prec in ("x3", "x6") else 0
    plan = fq.Plan.piecewise(a.h0, a.h1, fm, period=a.period, checkpoint_stride=16, precision=precision, tile_n=tile)
    L = plan.info.L
    f = torch.tensor(fm, device="cuda")
    W = torch.tensor(a.target, dtype=torch.complex128, device="cuda")
    ws = fq.workspace(fq.floquet_grad_workspace_size(plan.handle))
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(M, dtype=torch.float64, device="cuda")

    def step():
        fq.floquet_grad(plan.handle, f, W, loss, g, ws, stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if plan.check_status() != fq.FQ_OK:
        raise RuntimeError("device check fired during warm-up")
    per_step, total, clk = timed_loop(step, args.steps, stream, world, dist)
    value, total = job_throughput(total, args.steps, dist if world > 1 else None, "cuda")
    status_ok = plan.check_status() == fq.FQ_OK
    loss_value = float(loss.item())
    # end to end: plan from host arrays, f and W from pinned host memory, gradient and loss back
    f_h = torch.tensor(fm).pin_memory()
    w_h = torch.tensor(a.target, dtype=torch.complex128).pin_memory()
    g_h = torch.empty(M, dtype=torch.float64).pin_memory()
    l_h = torch.empty(1, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = fq.Plan.piecewise(a.h0, a.h1, fm, period=a.period, checkpoint_stride=16, precision=precision,
                               tile_n=tile)
        f.copy_(f_h, non_blocking=True)
        W.copy_(w_h, non_blocking=True)
        fq.floquet_grad(p2.handle, f, W, loss, g, ws, stream)
        g_h.copy_(g, non_blocking=True)
        l_h.copy_(loss, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        p2.close()
    e2e_value = world / statistics.median(e2e_times) if e2e_times else None
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    # products per gradient: the forward, recompute and adjoint chains (M L each) and the L dots
    # of every step; each is complex states x real operator, 4 N^3 useful flop
    useful = 4.0 * M * L * 4.0 * n ** 3
    issued = useful * SLICE_PRODUCTS[prec]
    avg = statistics.mean(per_step)
    achieved = useful / avg / 1e12
    if prec == "fp64":
        roofline = {"bound": "alu", "achieved": achieved, "peak": 1.19, "unit": "TFLOP/s", "frac": achieved / 1.19,
                    "traffic": None, "kernel": "k_adj_term / k_dot / dense_tile_f64",
                    "note": "FP64 SIMT; peak = the FP64 rate measured with the dense FP64 term kernel (1.19 TF)"}
    else:
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
                    "frac": achieved / peaks["bf16_sustained"], "traffic": None,
                    "kernel": "k_oz_real_term<*>" if prec == "ozaki" else "k_split_persist / k_split_term",
                    "issued_tflops": issued / avg / 1e12,
                    "issued_frac": issued / avg / 1e12 / peaks["bf16_sustained"],
                    "note": (f"achieved: useful 4 M L x 4 N^3 flop per gradient; issued: x {SLICE_PRODUCTS[prec]} "
                             "BF16 slice products; both over the gradient's CUDA-event time (every other kernel "
                             f"included); peak: {peaks['source']} sustained cuBLAS bf16")}
    accuracy = {"loss": loss_value}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, desc, (rl, rg, fs, Ts) = adjoint_oracle_sample(a)
        cpu = {"value": v, "unit": "grads/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}
        ps = fq.Plan.piecewise(a.h0, a.h1, fs, period=Ts, checkpoint_stride=16, precision=precision, tile_n=tile)
        ls, gs = ps.grad(torch.tensor(fs, device="cuda"), W)
        accuracy["sample_grad_max_err_vs_oracle"] = float(np.max(np.abs(gs.cpu().numpy() - rg)))
        accuracy["sample_grad_max_abs"] = float(np.max(np.abs(rg)))
        accuracy["sample_loss_err_vs_oracle"] = abs(float(ls.item()) - rl)
        accuracy["sample"] = desc
    line = {"metric": f"gradients/sec (gate fidelity, GOE N={n}, M={M} piecewise steps, checkpoints every 16)",
            "value": value, "unit": "grads/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"x3": "bf16 slices, f32 accumulate", "x6": "bf16 slices, f32 accumulate",
                      "ozaki": "bf16 slices, f64 states", "fp64": "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": f"adjoint: GOE N={n} (seeds 6, 7), Haar W (seed 8), f ~ N(1, 0.1^2) (seed 9), "
                                   f"M={M}, s=16, L={L}, {PREC_NAMES[prec]}",
                       "n": n, "steps": M, "chebyshev_L": L,
                       "l2": "working set larger than L2 (checkpoints and kept slices, > 1 GB)",
                       "parallelism": f"weak: {world} independent amplitude vectors"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "grads/s", "h2d_bytes_per_step": 2 * 8 * n * n + 8 * M + 16 * n * n,
                    "d2h_bytes_per_step": 8 * M + 8},
            "clocks": clk, "device_status_ok": status_ok, "accuracy": accuracy,
            "median_step_s": statistics.median(per_step), "per_step_s": per_step, "host": host_info()}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference_other(args):
    """--impl reference for goe4096 / adjoint: the oracle on a bounded sample, same metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import floquet_inputs as fi
    vals, desc = [], ""
    if args.workload == "batch":
        insts = fi.batch_scan()
        for _ in range(args.warmup):
            batch_oracle_sample(insts[:1], states=4, steps=1)
        for _ in range(args.steps):
            v, dt, desc = batch_oracle_sample(insts)
            vals.append(v)
        unit = "instances/s"
        metric = (f"instances/sec ({len(insts)}-instance dense GOE scan, N ~ U{{256..2048}}, M={BATCH_STEPS}, "
                  "one CUDA graph)")
        cfg = f"batched scan: {len(insts)} GOE instances, M={BATCH_STEPS}"
    elif args.workload in ("goe4096", "paper-table1"):
        paper = args.workload == "paper-table1"
        m = fi.config_goe_paper(args.n) if paper else fi.config_goe4096()
        terms = 50 if paper else 0
        for _ in range(args.warmup):
            dense_oracle_sample(m, states=8, steps=1, cheb_terms=terms)
        for _ in range(args.steps):
            v, dt, desc, _ = dense_oracle_sample(m, steps=2 if paper else 4, cheb_terms=terms)
            vals.append(v)
        unit = "U_T/s"
        if paper:
            metric = (f"U_T builds/sec (the paper's Table 1 timing run: GOE N={m.n} with unit-variance entries, "
                      f"f = cos(pi t), M={m.steps}, L=50, 6th-order Magnus)")
            cfg = f"paper Table 1: GOE N={m.n}, f=cos(pi t), M={m.steps}, L=50"
        else:
            metric = f"U_T builds/sec (dense GOE N={m.n}, M={m.steps})"
            cfg = f"dense GOE N={m.n} (seeds 3, 4), A=2, omega=2, M={m.steps}"
    else:
        a = fi.config_adjoint()
        for _ in range(args.warmup):
            adjoint_oracle_sample(a, steps=1)
        for _ in range(args.steps):
            v, dt, desc, _ = adjoint_oracle_sample(a)
            vals.append(v)
        metric = (f"gradients/sec (gate fidelity, GOE N={a.h0.shape[0]}, M={len(a.f)} piecewise steps, "
                  "checkpoints every 16)")
        unit = "grads/s"
        cfg = f"adjoint: GOE N={a.h0.shape[0]}, M={len(a.f)}"
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": cfg},
            "cpu_baseline": {"value": value, "unit": unit, "cores": os.cpu_count(), "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.ncu_case:
        run_ncu_case(a.ncu_case)
    elif a.impl == "reference":
        if a.workload in ("goe4096", "adjoint", "paper-table1", "batch"):
            run_reference_other(a)
        else:
            run_reference(a)
    elif a.workload in ("goe4096", "paper-table1"):
        run_dense(a)
    elif a.workload == "adjoint":
        run_adjoint(a)
    elif a.workload == "batch":
        run_batch(a)
    else:
        run_ours(a)

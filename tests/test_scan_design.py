"""The batched scan's schedule (csrc/scan.cu), checked on the CPU: the library's own unit table
(host-only hook fq_scan_table) expanded into the scan's global unit order, then run by a simulated
pool of CTAs that take units in order and wait exactly as the kernel does (its counters and their
targets).  An independent account of the data each unit reads and writes then checks that those
waits are enough: every term reads the Omega~ slices of its own step and the previous term's finished
state block, no block of Omega~ is overwritten while a term of the step that reads it is pending,
and every U_T store reads the last step's states.  The run must always finish (no unit waits on one
taken after it), for any number of CTAs and any unit durations."""
import ctypes
import heapq
import os
import random

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1508_07621_gb300", "libfloquet.so")
TERM, OMEGA, STORE = 0, 1, 2
BM, ROWS = 128, 16


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    import paper_1508_07621_gb300  # noqa: F401  (loads the library's dependencies)
    return ctypes.CDLL(LIB)


def table(lib, ns, Ls, steps, bn):
    cap = 4096
    seg = (ctypes.c_int * (4 * cap))()
    counts = (ctypes.c_int * 6)()
    arr = lambda v: (ctypes.c_int * len(v))(*v)
    k = lib.fq_scan_table(len(ns), arr(ns), arr(Ls), steps, bn, seg, cap, counts)
    assert k > 0
    segs = [tuple(seg[4 * i:4 * i + 4]) for i in range(k)]
    return segs, list(counts)


def expand(segs, counts, ns, Ls, steps, bn):
    """The global unit list as the kernel decodes it: (type, inst, m, p, t)."""
    npro, nstep, nend, upro, ustep, uend = counts
    parts = [(segs[:npro], upro), (segs[npro:npro + nstep], ustep), (segs[npro + nstep:], uend)]

    def units(part, total, m, region):
        out = []
        for k, (begin, typ, inst, p) in enumerate(part):
            end = part[k + 1][0] if k + 1 < len(part) else total
            for r in range(begin, end):
                if typ == TERM:
                    out.append((TERM, inst, m, p, r - begin))
                elif typ == OMEGA:
                    out.append((OMEGA, inst, 0 if region == 0 else m + 1, 0, p + r - begin))
                else:
                    out.append((STORE, inst, m, 0, r - begin))
        assert len(out) == total
        return out

    u = units(*parts[0], 0, 0)
    for m in range(steps):
        u += units(*parts[1], m, 1)
    return u + units(*parts[2], steps, 2)


def geometry(n, bn):
    np_ = -(-n // 128) * 128
    return dict(tiles_i=np_ // bn, tiles_j=-(-n // BM), nblk=np_ // ROWS)


def simulate(units, ns, Ls, steps, bn, workers, seed):
    rng = random.Random(seed)
    g = [geometry(n, bn) for n in ns]
    termcnt = {}     # (i, p, tj) -> finished tiles, across steps (the kernel counts 4 warps a tile)
    omegacnt = {}    # (i, parity) -> finished B units writing that Omega~ buffer
    done = set()
    # independent account of the data
    omega_ver = {}   # (i, buffer, block) -> step whose Omega~ rows the block holds
    block_ver = {}   # (i, tj) -> (m, p) of the last term finished on every tile of the block
    tiles_done = {}  # (i, m, p, tj) -> finished tiles
    reads_pending = {}  # (i, m) -> term units of step m not finished (they read buffer m % 2)
    for (typ, i, m, p, t) in units:
        if typ == TERM:
            reads_pending[(i, m)] = reads_pending.get((i, m), 0) + 1

    def ready(unit):
        typ, i, m, p, t = unit
        G = g[i]
        if typ == TERM:
            tj = t // G["tiles_i"]
            if omegacnt.get((i, m & 1), 0) < G["nblk"] * (m // 2 + 1):
                return False
            if p > 0:
                return termcnt.get((i, p - 1, tj), 0) >= G["tiles_i"] * (m + 1)
            if m > 0:
                return termcnt.get((i, Ls[i] - 1, tj), 0) >= G["tiles_i"] * m
            return True
        if typ == OMEGA:
            if m >= steps or m < 2:
                return True
            return all(termcnt.get((i, Ls[i] - 1, tj), 0) >= G["tiles_i"] * (m - 1) for tj in range(G["tiles_j"]))
        tj = (t * ROWS) // BM
        return termcnt.get((i, Ls[i] - 1, tj), 0) >= G["tiles_i"] * steps

    def start(unit):
        typ, i, m, p, t = unit
        G = g[i]
        if typ == TERM:
            tj = t // G["tiles_i"]
            assert all(omega_ver.get((i, m & 1, b)) == m for b in range(G["nblk"])), unit
            prev = (m, p - 1) if p > 0 else ((m - 1, Ls[i] - 1) if m > 0 else None)
            assert block_ver.get((i, tj)) == prev, (unit, block_ver.get((i, tj)))
        elif typ == OMEGA and m < steps:
            assert m < 2 or reads_pending.get((i, m - 2), 0) == 0, unit   # old readers finished
        elif typ == STORE:
            assert block_ver.get((i, (t * ROWS) // BM)) == (steps - 1, Ls[i] - 1), unit

    def finish(unit):
        typ, i, m, p, t = unit
        G = g[i]
        if typ == TERM:
            tj = t // G["tiles_i"]
            termcnt[(i, p, tj)] = termcnt.get((i, p, tj), 0) + 1
            key = (i, m, p, tj)
            tiles_done[key] = tiles_done.get(key, 0) + 1
            if tiles_done[key] == G["tiles_i"]:
                block_ver[(i, tj)] = (m, p)
            reads_pending[(i, m)] -= 1
        elif typ == OMEGA and m < steps:
            omegacnt[(i, m & 1)] = omegacnt.get((i, m & 1), 0) + 1
            omega_ver[(i, m & 1, t)] = m
        done.add(unit)

    nxt, clock, running, waiting = 0, 0.0, [], []
    idle = workers
    while True:
        while idle and nxt < len(units):      # idle CTAs take the next units, in order
            waiting.append(units[nxt])
            nxt += 1
            idle -= 1
        still = []
        for unit in waiting:                  # units whose waits are satisfied start now
            if ready(unit):
                start(unit)
                dur = rng.uniform(0.2, 2.0) * (3.0 if unit[0] == TERM else 1.0)
                heapq.heappush(running, (clock + dur, id(unit), unit))
            else:
                still.append(unit)
        waiting = still
        if not running:
            assert not waiting, f"stalled with {len(waiting)} waiting units"
            break
        clock, _, unit = heapq.heappop(running)
        finish(unit)
        idle += 1
    assert nxt == len(units) and len(done) == len(set(units))


CASES = [
    ([7, 129, 300, 260], [1, 2, 5, 8], 5, 64),
    ([7, 129, 300, 260], [1, 2, 5, 8], 5, 128),
    ([513, 40, 256], [3, 4, 3], 3, 128),
    ([200], [6], 1, 64),
    ([150, 389, 244], [17, 20, 12], 4, 128),
]


@pytest.mark.parametrize("ns,Ls,steps,bn", CASES)
def test_unit_table_covers_every_unit_once(lib, ns, Ls, steps, bn):
    """Per step: every instance's L terms, each on all its tiles once, and all its Omega~ blocks of
    the next step once; the prologue builds step 0's blocks, the end stores every state once."""
    segs, counts = table(lib, ns, Ls, steps, bn)
    units = expand(segs, counts, ns, Ls, steps, bn)
    assert len(set(units)) == len(units)
    for i, (n, L) in enumerate(zip(ns, Ls)):
        G = geometry(n, bn)
        for m in range(steps):
            for p in range(L):
                tiles = sorted(t for (ty, k, mm, pp, t) in units if ty == TERM and k == i and mm == m and pp == p)
                assert tiles == list(range(G["tiles_i"] * G["tiles_j"]))
        for m in range(steps + 1):
            blocks = sorted(t for (ty, k, mm, _, t) in units if ty == OMEGA and k == i and mm == m)
            assert blocks == list(range(G["nblk"]))
        stores = sorted(t for (ty, k, _, _, t) in units if ty == STORE and k == i)
        assert stores == list(range(-(-n // ROWS)))


@pytest.mark.parametrize("ns,Ls,steps,bn", CASES)
@pytest.mark.parametrize("workers", [1, 3, 11, 64])
def test_schedule_finishes_and_its_waits_protect_the_data(lib, ns, Ls, steps, bn, workers):
    segs, counts = table(lib, ns, Ls, steps, bn)
    units = expand(segs, counts, ns, Ls, steps, bn)
    simulate(units, ns, Ls, steps, bn, workers, seed=workers * 7919 + steps)


def test_table_rejects_what_the_kernel_cannot_run(lib):
    segs = (ctypes.c_int * 64)()
    counts = (ctypes.c_int * 6)()
    one = lambda v: (ctypes.c_int * 1)(v)
    assert lib.fq_scan_table(1, one(100), one(33), 4, 128, segs, 16, counts) == -1   # L > 32
    assert lib.fq_scan_table(1, one(100), one(4), 4, 96, segs, 16, counts) == -1     # tile width
    assert lib.fq_scan_table(1, one(100), one(4), 4, 128, segs, 1, counts) == -1     # capacity
    # 8320 units a step (16 x 16 tiles x 32 terms + 128 Omega~ blocks) over 10^6 steps: past the
    # kernel's 32-bit unit counter
    big = (ctypes.c_int * 1024)()
    assert lib.fq_scan_table(1, one(2048), one(32), 10 ** 6, 128, big, 256, counts) == -1
    assert lib.fq_scan_table(1, one(2048), one(32), 10 ** 5, 128, big, 256, counts) == 65

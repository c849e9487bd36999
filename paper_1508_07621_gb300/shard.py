"""Column split of one U_T over the ranks of a process group (§5, Fig. 2; the distribute and
gather parts of Algorithm 1).

The columns of U_T are independent: column j is the basis state e_j propagated over the period,
so rank r of P propagates its own block of columns with no exchange while they propagate, and
one all-gather assembles the result.  Blocks are ceil(N / P) columns; the last ranks take what
is left (possibly nothing), so every rank's block lands in a fixed slot of one gather buffer and
the gathered rows 0 .. N-1 are U_T in column-major order (row j = column j of U_T), the layout
the paper's master node collects.  The gather is in place: a rank's columns are written straight
into its slot of the buffer.

Host logic only (ranges, buffers, the collective); the propagation is the library's
floquet_build_UT_columns.
"""
from __future__ import annotations

from . import _binding as B


def column_block(n: int, rank: int, world: int) -> tuple[int, int, int]:
    """(j0, j1, bs): rank `rank` of `world` owns columns [j0, j1) of an n-column U_T; bs is the
    slot height ceil(n / world) shared by all ranks (j1 - j0 <= bs, possibly 0)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad split: n = {n}, rank {rank} of {world}")
    bs = -(-n // world)
    j0 = min(rank * bs, n)
    return j0, min(j0 + bs, n), bs


def gather_buffer(n: int, world: int, device="cuda"):
    """The all-gather buffer: world slots of ceil(n / world) rows of n complex128 entries."""
    import torch
    return torch.empty((world * (-(-n // world)), n), dtype=torch.complex128, device=device)


def slot(buf, rank: int, world: int):
    """This rank's rows of the gather buffer (a view)."""
    bs = buf.shape[0] // world
    return buf[rank * bs:(rank + 1) * bs]


def all_gather_columns(buf, n: int, dist):
    """In-place all-gather of every rank's slot; returns rows 0 .. n-1 of the buffer (U_T
    column-major: row j = column j).  Rows past a rank's real columns carry whatever its slot
    held; they sit at the buffer's end, beyond row n - 1."""
    import torch
    rank, world = dist.get_rank(), dist.get_world_size()
    dist.all_gather_into_tensor(torch.view_as_real(buf), torch.view_as_real(slot(buf, rank, world)))
    return buf[:n]


def columns_workspace(plan, world: int):
    """Workspace for this plan's largest column block (the same on every rank)."""
    from .api import workspace
    bs = -(-plan.n // world)
    return workspace(B.floquet_columns_workspace_size(plan.handle, max(bs, 1)))


def build_ut_sharded(plan, dist, buf=None, ws=None, stream=None):
    """One U_T built by all ranks of `dist`: each propagates its column block into its slot
    (floquet_build_UT_columns), then one all-gather.  Every rank holds the same plan.  Returns
    U_T column-major (row j = column j of U_T, complex128, on the current device); use `.mT` for
    U_T itself as a strided view."""
    rank, world = dist.get_rank(), dist.get_world_size()
    n = plan.n
    if buf is None:
        buf = gather_buffer(n, world)
    if ws is None:
        ws = columns_workspace(plan, world)
    j0, j1, _ = column_block(n, rank, world)
    if j1 > j0:
        B.floquet_build_UT_columns(plan.handle, j0, j1 - j0, slot(buf, rank, world), ws, stream)
    return all_gather_columns(buf, n, dist)

"""Convenience layer over the binding: a plan handle that frees itself, and torch-allocated
outputs/workspaces.  Still marshalling only - every computation is a libfloquet.so call."""
from __future__ import annotations

import math

from . import _binding as B


def workspace(nbytes: int, device="cuda"):
    """Caller-owned device workspace (torch allocation, 256-byte aligned by the allocator)."""
    import torch
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


class Plan:
    """Owns an fq_plan*; destroyed on close() / garbage collection."""

    def __init__(self, problem, keepalive):
        self._keep = keepalive
        self.handle = B.floquet_plan_create(problem)
        self.info = B.floquet_plan_get_info(self.handle)
        self.n = self.info.n

    # ---------------------------------------------------------------- constructors
    @classmethod
    def dense(cls, h0, h1, *, omega, f_ac, steps, f_dc=0.0, phi0=0.0, period=None, precision=B.FQ_FP64,
              cheb_tol=0.0, e_min=0.0, e_max=0.0, tile_n=0, magnus_order=0, kernel=B.FQ_KERNEL_AUTO,
              cheb_terms=0, tile_k=0):
        n = h0.shape[0]
        T = period if period is not None else 2.0 * math.pi / omega
        prob, keep = B.make_problem(n, B.FQ_DENSE, h0, h1, T, steps, f_dc=f_dc, f_ac=f_ac, omega=omega,
                                    phi0=phi0, precision=precision, cheb_tol=cheb_tol, e_min=e_min, e_max=e_max,
                                    tile_n=tile_n, magnus_order=magnus_order, kernel=kernel, cheb_terms=cheb_terms,
                                    tile_k=tile_k)
        return cls(prob, keep)

    @classmethod
    def tridiag(cls, h0_diag, h0_off, h1_diag, *, omega, f_ac, steps, f_dc=0.0, phi0=0.0, period=None,
                precision=None, kernel=B.FQ_KERNEL_AUTO, cheb_tol=0.0, e_min=0.0, e_max=0.0, magnus_order=0):
        """precision defaults to FQ_FP32 (FQ_FP64 for magnus_order 6, the only one it runs in)."""
        n = h0_diag.shape[0]
        T = period if period is not None else 2.0 * math.pi / omega
        if precision is None:
            precision = B.FQ_FP64 if magnus_order == 6 else B.FQ_FP32
        prob, keep = B.make_problem(n, B.FQ_TRIDIAG, h0_diag, h1_diag, T, steps, h0_off=h0_off, f_dc=f_dc,
                                    f_ac=f_ac, omega=omega, phi0=phi0, precision=precision, kernel=kernel,
                                    cheb_tol=cheb_tol, e_min=e_min, e_max=e_max, magnus_order=magnus_order)
        return cls(prob, keep)

    @classmethod
    def piecewise(cls, h0, h1, f_steps, *, period, precision=B.FQ_FP64, checkpoint_stride=16, cheb_tol=0.0,
                  tile_n=0):
        n = h0.shape[0]
        prob, keep = B.make_problem(n, B.FQ_DENSE, h0, h1, period, len(f_steps), drive_kind=B.FQ_DRIVE_PIECEWISE,
                                    f_steps=f_steps, precision=precision, checkpoint_stride=checkpoint_stride,
                                    cheb_tol=cheb_tol, tile_n=tile_n)
        return cls(prob, keep)

    # ---------------------------------------------------------------- calls
    def workspace_size(self, ncols=None) -> int:
        return B.floquet_workspace_size(self.handle, self.n if ncols is None else ncols)

    def build_UT(self, out=None, ws=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.complex128, device="cuda")
        if ws is None:
            ws = workspace(self.workspace_size())
        B.floquet_build_UT(self.handle, out, ws, stream)
        return out

    def propagate(self, x0, m_begin=0, m_end=None, out=None, ws=None, stream=None):
        import torch
        m_end = self.info.steps if m_end is None else m_end
        ncols = x0.shape[0]
        if out is None:
            out = torch.empty_like(x0)
        if ws is None:
            ws = workspace(self.workspace_size(ncols))
        B.floquet_propagate(self.handle, x0, out, ncols, m_begin, m_end, ws, stream)
        return out

    def grad(self, f, W, ws=None, stream=None):
        """(loss, dL/df) of L = 1 - |Tr(W^+ U_T)|^2 / N^2 for the piecewise amplitudes f (device tensors)."""
        import torch
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty(self.info.steps, dtype=torch.float64, device="cuda")
        if ws is None:
            ws = workspace(B.floquet_grad_workspace_size(self.handle))
        B.floquet_grad(self.handle, f, W, loss, g, ws, stream)
        return loss, g

    def average_observable(self, states, a0=1.0, a1=0.0, s_drive=1.0, stream=None):
        """<A>_T of every row of `states` (complex128, ncols x N) for A(t) = a0 H0 + (a1 + s f(t)) H1."""
        import torch
        ncols = states.shape[0]
        out = torch.empty(ncols, dtype=torch.float64, device="cuda")
        ws = workspace(B.floquet_observable_workspace_size(self.handle, ncols))
        B.floquet_average_observable(self.handle, states, ncols, a0, a1, s_drive, out, ws, stream)
        return out

    def autotune(self, ws=None, stream=None) -> int:
        if ws is None:
            ws = workspace(self.workspace_size())
        return B.floquet_autotune(self.handle, ws, stream)

    def check_status(self, stream=None) -> int:
        return B.floquet_check_status(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            B.floquet_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_FIDELITY_FN = None


def _fidelity_function():
    """torch.autograd.Function whose forward and backward are one floquet_grad call: the loss
    and dL/df come out of the same forward sweep plus adjoint chain, and backward scales the
    kept gradient by the incoming cotangent."""
    global _FIDELITY_FN
    if _FIDELITY_FN is None:
        import torch

        class FidelityLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, f, plan, W):
                loss, g = plan.grad(f.detach().to(torch.float64).contiguous(), W)
                ctx.save_for_backward(g)
                return loss[0]

            @staticmethod
            def backward(ctx, gout):
                (g,) = ctx.saved_tensors
                return gout * g, None, None

        _FIDELITY_FN = FidelityLoss
    return _FIDELITY_FN


def fidelity_loss(plan, f, W):
    """Gate-fidelity loss L(f) = 1 - |Tr(W^+ U_T(f))|^2 / N^2 as a differentiable torch scalar of
    the piecewise amplitudes f (float64 device tensor of length M; plan from Plan.piecewise, W an
    N x N complex128 device tensor).  Its gradient is the library's adjoint (floquet_grad)."""
    return _fidelity_function().apply(f, plan, W)


def unitarity_defect(U, cols=None, stream=None):
    """(max |U^+U - 1|, Frobenius / sqrt(k)) over the listed columns (all if None)."""
    n = U.shape[0]
    k = n if cols is None else cols.numel()
    ws = workspace(B.floquet_defect_workspace_size(n))  # sized for all n rows, so enough for any k <= n
    return B.floquet_unitarity_defect(U, n, cols, k, ws, stream)


def floquet_states(U, period):
    """Quasienergies eps (Eq. 5, eps = theta/T, theta = -arg(lambda) in [-pi, pi), ascending) and
    Floquet states (rows, unit norm, on U's device) of U_T by the library's host solver
    (floquet_quasienergies) - outside the timed path.  Returns (eps as a numpy array, states)."""
    import torch
    eps, v = B.floquet_quasienergies(U.detach().cpu().numpy(), period, states=True)
    return eps, torch.from_numpy(v).to(U.device)


def floquet_analysis(plan, U=None):
    """The paper's post-processing (§3 last paragraph, §7): Floquet states of U_T (library host
    solver), their period-averaged energies <H(t)>_T from a second propagation round (Eq. 17, on
    the library), and the states sorted by that energy.  Returns (avg_energy, eps, states), sorted
    ascending in avg_energy; states are rows (complex128, device)."""
    import numpy as np
    import torch
    if U is None:
        U = plan.build_UT()
    eps, states = floquet_states(U, plan.info.steps * plan.info.h)
    avg = plan.average_observable(states, 1.0, 0.0, 1.0).cpu().numpy()
    order = np.argsort(avg, kind="stable")
    idx = torch.from_numpy(order).to(states.device)
    return avg[order], eps[order], states.index_select(0, idx)


def overlap_phase_error(plan, U_fine, stream=None):
    """Overlap phase error of Eq. 20 for the chain of `plan` (step h): with (phi~, eps~) the
    Floquet states of U_fine, the U_T of the same drive at step h/2, Sigma_mu =
    |1 - e^{i eps~_mu T} <phi~_mu| U_T |phi~_mu>| (floquet_overlap_phase_error: the chain and the
    overlaps on the device).  Returns (eps~ ascending, Sigma in that order) as numpy arrays."""
    import torch
    T = plan.info.steps * plan.info.h
    eps, states = floquet_states(U_fine, T)
    n = states.shape[0]
    d_eps = torch.from_numpy(eps).to(states.device)
    sigma = torch.empty(n, dtype=torch.float64, device=states.device)
    ws = workspace(B.floquet_overlap_workspace_size(plan.handle, n))
    B.floquet_overlap_phase_error(plan.handle, states, n, d_eps, sigma, ws, stream)
    return eps, sigma.cpu().numpy()

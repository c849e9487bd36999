"""ctypes binding of libfloquet.so: argument marshalling only.

Every function here has the name of the C entry point it calls and only converts
arguments (torch tensors -> device pointers, torch streams -> cudaStream_t, Python numbers ->
C types).  All computation happens in the library's CUDA kernels and host planner; there is
no fallback: if libfloquet.so is missing, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfloquet.so")

FQ_OK, FQ_EINVAL, FQ_ENOMEM, FQ_ECUDA, FQ_EBOUND, FQ_ETIMEOUT, FQ_EUNSUPPORTED = range(7)
FQ_DENSE, FQ_TRIDIAG = 0, 1
FQ_FP64, FQ_FP32, FQ_BF16X3, FQ_BF16X6, FQ_DF32, FQ_OZAKI = 0, 1, 2, 3, 4, 5
FQ_DRIVE_COS, FQ_DRIVE_PIECEWISE = 0, 1
FQ_KERNEL_AUTO, FQ_KERNEL_STREAM, FQ_KERNEL_RESIDENT, FQ_KERNEL_TILED, FQ_KERNEL_BAND = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "FQ_OK", 1: "FQ_EINVAL", 2: "FQ_ENOMEM", 3: "FQ_ECUDA", 4: "FQ_EBOUND",
                5: "FQ_ETIMEOUT", 6: "FQ_EUNSUPPORTED"}

_dp = ctypes.POINTER(ctypes.c_double)


class fq_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("format", ctypes.c_int32),
                ("h0", _dp), ("h0_off", _dp), ("h1", _dp),
                ("period", ctypes.c_double), ("steps", ctypes.c_int32), ("drive_kind", ctypes.c_int32),
                ("f_dc", ctypes.c_double), ("f_ac", ctypes.c_double), ("omega", ctypes.c_double),
                ("phi0", ctypes.c_double), ("f_steps", _dp), ("cheb_tol", ctypes.c_double),
                ("e_min", ctypes.c_double), ("e_max", ctypes.c_double), ("precision", ctypes.c_int32),
                ("checkpoint_stride", ctypes.c_int32), ("kernel", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("magnus_order", ctypes.c_int32), ("cheb_terms", ctypes.c_int32), ("tile_k", ctypes.c_int32)]


class fq_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("steps", ctypes.c_int32), ("L", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("format", ctypes.c_int32), ("drive_kind", ctypes.c_int32),
                ("h", ctypes.c_double), ("e_min", ctypes.c_double), ("e_max", ctypes.c_double),
                ("beta", ctypes.c_double), ("delta_e", ctypes.c_double), ("R", ctypes.c_double)]


class fq_report(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("defect_columns", ctypes.c_int32), ("R", ctypes.c_double),
                ("e_min", ctypes.c_double), ("e_max", ctypes.c_double), ("beta", ctypes.c_double),
                ("delta_e", ctypes.c_double), ("defect_max", ctypes.c_double), ("defect_fro", ctypes.c_double),
                ("build_ms", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_1508_07621_gb300.build.build() "
                      "(nvcc for sm_103a) first - there is no CPU fallback")
lib = ctypes.CDLL(LIB_PATH)

_vp, _sz, _i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32
_SIGS = {
    "floquet_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(fq_problem)]),
    "floquet_plan_destroy": (None, [_vp]),
    "floquet_plan_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(fq_plan_info)]),
    "floquet_plan_inspect": (ctypes.c_int, [ctypes.POINTER(fq_problem), ctypes.POINTER(fq_plan_info), _dp, _i32]),
    "floquet_workspace_size": (_sz, [_vp, _i32]),
    "floquet_build_UT": (ctypes.c_int, [_vp, _vp, _vp, _sz, _vp]),
    "floquet_propagate": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _sz, _vp]),
    "floquet_build_UT_report": (ctypes.c_int, [_vp, _vp, _vp, _sz, _vp, _i32, ctypes.POINTER(fq_report)]),
    "floquet_columns_workspace_size": (_sz, [_vp, _i32]),
    "floquet_build_UT_columns": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _sz, _vp]),
    "floquet_defect_workspace_size": (_sz, [_i32]),
    "floquet_unitarity_defect": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _sz, _vp, _dp, _dp]),
    "floquet_grad_workspace_size": (_sz, [_vp]),
    "floquet_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "floquet_selftest_wait": (ctypes.c_int, [_vp, ctypes.c_int64, _vp]),
    "floquet_probe_fp32": (ctypes.c_int, [_i32, _i32, _vp, ctypes.c_int64, _vp, _dp]),
    "floquet_quasienergies": (ctypes.c_int, [_vp, _i32, ctypes.c_double, _dp, _vp]),
    "floquet_check_status": (ctypes.c_int, [_vp, _vp]),
    "floquet_build_UT_static": (ctypes.c_int, [ctypes.POINTER(fq_problem), _vp, _vp]),
    "floquet_batch_workspace_size": (_sz, [ctypes.POINTER(_vp), _i32]),
    "floquet_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp),
                                            _vp, _sz, _i32]),
    "floquet_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "floquet_batch_destroy": (None, [_vp]),
    "floquet_autotune": (ctypes.c_int, [_vp, _vp, _sz, _vp, ctypes.POINTER(_i32)]),
    "floquet_observable_workspace_size": (_sz, [_vp, _i32]),
    "floquet_average_observable": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, _vp, _vp, _sz, _vp]),
    "floquet_overlap_workspace_size": (_sz, [_vp, _i32]),
    "floquet_overlap_phase_error": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _sz, _vp]),
    "floquet_kernel_timing": (ctypes.c_int, [_vp, _i32]),
    "floquet_kernel_time": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), _dp, ctypes.c_char_p, _i32]),
    "floquet_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class FloquetError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str | None = None):
        if msg is None:
            msg = lib.floquet_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str):
    if status != FQ_OK:
        raise FloquetError(status, where)


def _dev(t, dtype, count: int, what: str, where: str):
    """Device pointer of `t` once it is known to be a contiguous CUDA tensor on the current
    device, of `dtype` (None: any) and with at least `count` elements; None -> NULL.  The library
    takes raw device pointers on trust, so a host, strided, mistyped or short tensor is refused
    here with FQ_EINVAL instead of reaching a kernel."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FloquetError(FQ_EINVAL, where, f"{what} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise FloquetError(FQ_EINVAL, where, f"{what} is on {t.device}, the current device is "
                           f"cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise FloquetError(FQ_EINVAL, where, f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise FloquetError(FQ_EINVAL, where, f"{what} must be {dtype} (got {t.dtype})")
    if t.numel() < count:
        raise FloquetError(FQ_EINVAL, where, f"{what} has {t.numel()} elements, the call needs {count}")
    return ctypes.c_void_p(t.data_ptr())


def _ws(ws, where: str):
    """(pointer, bytes) of a workspace tensor (any dtype; its size is checked by the library)."""
    return _dev(ws, None, 0, "workspace", where), (ws.numel() * ws.element_size() if ws is not None else 0)


def _c128():
    import torch
    return torch.complex128


def _f64():
    import torch
    return torch.float64


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _darr(a):
    import numpy as np
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr, arr.ctypes.data_as(_dp)


def make_problem(n, fmt, h0, h1, period, steps, h0_off=None, drive_kind=FQ_DRIVE_COS, f_dc=0.0, f_ac=0.0,
                 omega=1.0, phi0=0.0, f_steps=None, cheb_tol=0.0, e_min=0.0, e_max=0.0,
                 precision=FQ_FP64, checkpoint_stride=0, kernel=FQ_KERNEL_AUTO, tile_n=0, magnus_order=0,
                 cheb_terms=0, tile_k=0):
    """Builds an fq_problem; returns (struct, keepalive) - the host arrays must outlive the call."""
    a0, p0 = _darr(h0)
    a1, p1 = _darr(h1)
    ao, po = _darr(h0_off)
    af, pf = _darr(f_steps)
    # the library reads these host arrays to the sizes the problem implies
    nop = n * n if fmt == FQ_DENSE else n if fmt == FQ_TRIDIAG else 0
    for arr, need, what in ((a0, nop, "h0"), (a1, nop, "h1"), (ao, n - 1 if fmt == FQ_TRIDIAG else 0, "h0_off"),
                            (af, steps if drive_kind == FQ_DRIVE_PIECEWISE else 0, "f_steps")):
        if arr is not None and arr.size < need:
            raise ValueError(f"make_problem: {what} has {arr.size} values, the problem needs {need}")
    prob = fq_problem(n, fmt, p0, po, p1, period, steps, drive_kind, f_dc, f_ac, omega, phi0, pf, cheb_tol,
                      e_min, e_max, precision, checkpoint_stride, kernel, tile_n, magnus_order, cheb_terms, tile_k)
    return prob, (a0, a1, ao, af)


def floquet_plan_create(problem) -> int:
    plan = _vp()
    _check(lib.floquet_plan_create(ctypes.byref(plan), ctypes.byref(problem)), "floquet_plan_create")
    return plan.value


def floquet_plan_destroy(plan: int) -> None:
    lib.floquet_plan_destroy(_vp(plan))


def floquet_plan_get_info(plan: int) -> fq_plan_info:
    info = fq_plan_info()
    _check(lib.floquet_plan_get_info(_vp(plan), ctypes.byref(info)), "floquet_plan_get_info")
    return info


def floquet_plan_inspect(problem, cap: int = 4096):
    import numpy as np
    info = fq_plan_info()
    coeffs = np.zeros(cap)
    _check(lib.floquet_plan_inspect(ctypes.byref(problem), ctypes.byref(info), coeffs.ctypes.data_as(_dp), cap),
           "floquet_plan_inspect")
    return info, coeffs[: info.L + 1].copy()


def floquet_workspace_size(plan: int, ncols: int) -> int:
    return int(lib.floquet_workspace_size(_vp(plan), ncols))


def floquet_build_UT(plan: int, U, ws, stream=None) -> None:
    w = "floquet_build_UT"
    n = floquet_plan_get_info(plan).n
    pu = _dev(U, _c128(), n * n, "U", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_build_UT(_vp(plan), pu, pw, nb, _stream(stream)), w)


def floquet_build_UT_report(plan: int, U, ws, defect_columns: int = 64, stream=None) -> fq_report:
    """floquet_build_UT plus its report (planning results, sampled unitarity defect, device time)."""
    w = "floquet_build_UT_report"
    n = floquet_plan_get_info(plan).n
    pu = _dev(U, _c128(), n * n, "U", w)
    pw, nb = _ws(ws, w)
    rep = fq_report()
    _check(lib.floquet_build_UT_report(_vp(plan), pu, pw, nb, _stream(stream), int(defect_columns),
                                       ctypes.byref(rep)), w)
    return rep


def floquet_kernel_timing(plan: int, enable: bool) -> None:
    """Switches the event timing of the chain's step kernel on or off (and clears its record)."""
    _check(lib.floquet_kernel_timing(_vp(plan), 1 if enable else 0), "floquet_kernel_timing")


def floquet_kernel_time(plan: int) -> tuple[int, float, str]:
    """(launches, total milliseconds, kernel name) recorded since the last read."""
    n = _i32(0)
    ms = ctypes.c_double(0.0)
    buf = ctypes.create_string_buffer(64)
    _check(lib.floquet_kernel_time(_vp(plan), ctypes.byref(n), ctypes.byref(ms), buf, 64), "floquet_kernel_time")
    return int(n.value), float(ms.value), buf.value.decode()


def floquet_propagate(plan: int, X0, X, ncols: int, m_begin: int, m_end: int, ws, stream=None) -> None:
    w = "floquet_propagate"
    n = floquet_plan_get_info(plan).n
    need = max(int(ncols), 0) * n
    px0, px = _dev(X0, _c128(), need, "X0", w), _dev(X, _c128(), need, "X", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_propagate(_vp(plan), px0, px, ncols, m_begin, m_end, pw, nb, _stream(stream)), w)


def floquet_defect_workspace_size(n: int) -> int:
    return int(lib.floquet_defect_workspace_size(n))


def floquet_unitarity_defect(U, n: int, cols, k: int, ws, stream=None):
    import torch
    w = "floquet_unitarity_defect"
    mx, fro = ctypes.c_double(), ctypes.c_double()
    pu = _dev(U, _c128(), max(int(n), 0) ** 2, "U", w)
    pc = _dev(cols, torch.int32, max(int(k), 0), "cols", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_unitarity_defect(pu, n, pc, k, pw, nb, _stream(stream), ctypes.byref(mx), ctypes.byref(fro)), w)
    return mx.value, fro.value


def floquet_grad_workspace_size(plan: int) -> int:
    return int(lib.floquet_grad_workspace_size(_vp(plan)))


def floquet_grad(plan: int, f, W, loss, grad, ws, stream=None) -> None:
    w = "floquet_grad"
    info = floquet_plan_get_info(plan)
    pf, pW = _dev(f, _f64(), info.steps, "f", w), _dev(W, _c128(), info.n * info.n, "W", w)
    pl, pg = _dev(loss, _f64(), 1, "loss", w), _dev(grad, _f64(), info.steps, "grad", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_grad(_vp(plan), pf, pW, pl, pg, pw, nb, _stream(stream)), w)


def floquet_build_UT_static(problem, U, stream=None) -> None:
    """No-allocation U_T (resident FP32 tridiagonal chain, static device scratch); see floquet.h."""
    w = "floquet_build_UT_static"
    _check(lib.floquet_build_UT_static(ctypes.byref(problem), _dev(U, _c128(), max(problem.n, 0) ** 2, "U", w),
                                       _stream(stream)), w)


def floquet_batch_workspace_size(plans) -> int:
    arr = (_vp * len(plans))(*plans)
    return int(lib.floquet_batch_workspace_size(arr, len(plans)))


def floquet_batch_create(plans, outputs, ws, lanes: int = 0) -> int:
    """One CUDA graph for the U_T builds of all plans; outputs[i]: N_i x N_i complex128 tensors.
    lanes = 0: one persistent launch over work units where the plans allow it (else 8 lanes)."""
    w = "floquet_batch_create"
    if len(outputs) != len(plans):
        raise FloquetError(FQ_EINVAL, w, f"{len(plans)} plans but {len(outputs)} outputs")
    arr = (_vp * len(plans))(*plans)
    outs = (_vp * len(outputs))(*[_dev(o, _c128(), floquet_plan_get_info(p).n ** 2, f"outputs[{i}]", w)
                                  for i, (p, o) in enumerate(zip(plans, outputs))])
    b = _vp()
    pw, nb = _ws(ws, w)
    _check(lib.floquet_batch_create(ctypes.byref(b), arr, len(plans), outs, pw, nb, lanes), w)
    return b.value


def floquet_batch_launch(batch: int, stream=None) -> None:
    _check(lib.floquet_batch_launch(_vp(batch), _stream(stream)), "floquet_batch_launch")


def floquet_batch_destroy(batch: int) -> None:
    lib.floquet_batch_destroy(_vp(batch))


def floquet_autotune(plan: int, ws, stream=None) -> int:
    tile = _i32()
    pw, nb = _ws(ws, "floquet_autotune")
    _check(lib.floquet_autotune(_vp(plan), pw, nb, _stream(stream), ctypes.byref(tile)), "floquet_autotune")
    return tile.value


def floquet_observable_workspace_size(plan: int, ncols: int) -> int:
    return int(lib.floquet_observable_workspace_size(_vp(plan), ncols))


def floquet_average_observable(plan: int, X0, ncols: int, a0: float, a1: float, s_drive: float, out, ws,
                               stream=None) -> None:
    w = "floquet_average_observable"
    n = floquet_plan_get_info(plan).n
    px = _dev(X0, _c128(), max(int(ncols), 0) * n, "X0", w)
    po = _dev(out, _f64(), max(int(ncols), 0), "out", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_average_observable(_vp(plan), px, ncols, a0, a1, s_drive, po, pw, nb, _stream(stream)), w)


def floquet_columns_workspace_size(plan: int, ncols: int) -> int:
    return int(lib.floquet_columns_workspace_size(_vp(plan), ncols))


def floquet_build_UT_columns(plan: int, j0: int, ncols: int, out, ws, stream=None) -> None:
    w = "floquet_build_UT_columns"
    n = floquet_plan_get_info(plan).n
    po = _dev(out, _c128(), max(int(ncols), 0) * n, "out", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_build_UT_columns(_vp(plan), j0, ncols, po, pw, nb, _stream(stream)), w)


def floquet_overlap_workspace_size(plan: int, ncols: int) -> int:
    return int(lib.floquet_overlap_workspace_size(_vp(plan), ncols))


def floquet_overlap_phase_error(plan: int, states, ncols: int, eps, sigma, ws, stream=None) -> None:
    w = "floquet_overlap_phase_error"
    n = floquet_plan_get_info(plan).n
    ps = _dev(states, _c128(), max(int(ncols), 0) * n, "states", w)
    pe = _dev(eps, _f64(), max(int(ncols), 0), "eps", w)
    po = _dev(sigma, _f64(), max(int(ncols), 0), "sigma", w)
    pw, nb = _ws(ws, w)
    _check(lib.floquet_overlap_phase_error(_vp(plan), ps, ncols, pe, po, pw, nb, _stream(stream)), w)


def floquet_check_status(plan: int, stream=None) -> int:
    return int(lib.floquet_check_status(_vp(plan), _stream(stream)))


def floquet_quasienergies(u, period: float, states: bool = True):
    """(eps ascending, Floquet states as rows or None) of the host complex128 N x N array u by
    the library's host Schur solver."""
    import numpy as np
    u = np.ascontiguousarray(u, dtype=np.complex128)
    if u.ndim != 2 or u.shape[0] != u.shape[1]:
        raise FloquetError(FQ_EINVAL, "floquet_quasienergies", f"U must be a square matrix (got shape {u.shape})")
    n = u.shape[0]
    eps = np.empty(n)
    out = np.empty((n, n), dtype=np.complex128) if states else None
    _check(lib.floquet_quasienergies(u.ctypes.data_as(_vp), n, float(period), eps.ctypes.data_as(_dp),
                                     out.ctypes.data_as(_vp) if states else None), "floquet_quasienergies")
    return eps, out


def floquet_selftest_wait(plan: int, cycles: int, stream=None) -> None:
    _check(lib.floquet_selftest_wait(_vp(plan), int(cycles), _stream(stream)), "floquet_selftest_wait")


def floquet_probe_fp32(packed: bool, iters: int, out, stream=None) -> float:
    """Enqueues the FP32 rate probe on `stream` (out: float32 CUDA tensor of >= 256 elements);
    returns the launch's flop count."""
    w = "floquet_probe_fp32"
    import torch
    fl = ctypes.c_double()
    _check(lib.floquet_probe_fp32(1 if packed else 0, int(iters), _dev(out, torch.float32, 256, "out", w),
                                  out.numel(), _stream(stream), ctypes.byref(fl)), w)
    return fl.value


def floquet_last_error() -> str:
    return lib.floquet_last_error().decode(errors="replace")

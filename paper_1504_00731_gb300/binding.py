"""Thin ctypes binding of the C ABI in include/weno_theta.h.

Argument marshalling only: every step of the computation runs in the CUDA library
``libweno_theta.so`` (built in-tree by ``paper_1504_00731_gb300.build``).  Arrays may be
torch tensors (CUDA or CPU, float64, contiguous) or numpy float64 arrays; CUDA tensors
run on torch's current stream unless a stream is given.  Importing this module does not
need a GPU; calling an entry point without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libweno_theta.so")

WT_OK, WT_ERR_ARG, WT_ERR_UNSUPPORTED, WT_ERR_CUDA, WT_ERR_NONPHYSICAL, WT_ERR_TIMEOUT, WT_ERR_WORKSPACE = (
    0, -1, -2, -3, -4, -5, -6)
WT_FLUX_ADVECTION, WT_FLUX_BURGERS, WT_FLUX_EULER1D, WT_FLUX_EULER2D = 0, 1, 2, 3
WT_BC_PERIODIC, WT_BC_OUTFLOW, WT_BC_REFLECTIVE = 0, 1, 2
WT_MODE_FAST, WT_MODE_STRICT = 0, 1
WT_LAUNCH_AUTO, WT_LAUNCH_STAGES = 0, 1
_M = {WT_FLUX_ADVECTION: 1, WT_FLUX_BURGERS: 1, WT_FLUX_EULER1D: 3, WT_FLUX_EULER2D: 4}

# every entry point declared in include/weno_theta.h
EXPORTED = (
    "wt_workspace_bytes",
    "weno_theta_rhs",
    "weno_theta_step",
    "weno_theta_step_batched",
    "wt_adjoint_workspace_bytes",
    "weno_theta_adjoint",
    "weno_theta_rhs_noalloc",
    "wt_selftest_wait",
    "wt_last_error",
)


class WtProblem(ctypes.Structure):
    _fields_ = [
        ("flux", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("adv_speed", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("alpha_R", ctypes.c_double),
        ("bc_lo", ctypes.c_int32 * 2),
        ("bc_hi", ctypes.c_int32 * 2),
        ("mode", ctypes.c_int32),
        ("launch", ctypes.c_int32),
        ("gravity", ctypes.c_double),
    ]


class WtGrid(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("n", ctypes.c_int64 * 2),
        ("lo", ctypes.c_double * 2),
        ("hi", ctypes.c_double * 2),
    ]


class WtSegment(ctypes.Structure):
    _fields_ = [
        ("offset", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("lo", ctypes.c_double),
        ("hi", ctypes.c_double),
        ("bc_lo", ctypes.c_int32),
        ("bc_hi", ctypes.c_int32),
    ]


class WenoThetaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"status {status}: {message}")
        self.status = status


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1504_00731_gb300.build.build_library()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.wt_workspace_bytes.argtypes = [P(WtProblem), P(WtGrid), ctypes.c_int64, ctypes.c_int32]
    L.wt_workspace_bytes.restype = ctypes.c_size_t
    L.weno_theta_rhs.argtypes = [P(WtProblem), P(WtGrid), vp, vp, vp, ctypes.c_size_t, vp]
    L.weno_theta_rhs.restype = ctypes.c_int
    L.weno_theta_step.argtypes = [P(WtProblem), P(WtGrid), vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int64), vp, ctypes.c_size_t, vp]
    L.weno_theta_step.restype = ctypes.c_int
    L.weno_theta_step_batched.argtypes = [P(WtProblem), P(WtSegment), ctypes.c_int32, vp, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_int64, vp, vp, vp, ctypes.c_size_t, vp]
    L.weno_theta_step_batched.restype = ctypes.c_int
    L.wt_adjoint_workspace_bytes.argtypes = [P(WtProblem), P(WtGrid), ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
    L.wt_adjoint_workspace_bytes.restype = ctypes.c_size_t
    L.weno_theta_adjoint.argtypes = [P(WtProblem), P(WtGrid), ctypes.c_int32, vp, ctypes.c_double, ctypes.c_int64,
                                     ctypes.c_int32, vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.weno_theta_adjoint.restype = ctypes.c_int
    L.weno_theta_rhs_noalloc.argtypes = [P(WtProblem), P(WtGrid), vp, vp, vp]
    L.weno_theta_rhs_noalloc.restype = ctypes.c_int
    L.wt_selftest_wait.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, ctypes.c_size_t, vp]
    L.wt_selftest_wait.restype = ctypes.c_int
    L.wt_last_error.argtypes = []
    L.wt_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def last_error() -> str:
    m = lib().wt_last_error()
    return m.decode() if m else ""


def _check(status):
    if status != WT_OK:
        raise WenoThetaError(status, last_error())


def problem(flux, gamma=1.4, adv_speed=1.0, eps=1e-10, alpha_R=50.0, bc=WT_BC_PERIODIC, bc_y=None,
            mode=WT_MODE_FAST, gravity=0.0, launch=0) -> WtProblem:
    p = WtProblem()
    p.flux = flux
    p.m = _M[flux]
    p.gamma = gamma
    p.adv_speed = adv_speed
    p.eps = eps
    p.alpha_R = alpha_R
    lo, hi = (bc, bc) if isinstance(bc, int) else bc
    by = bc if bc_y is None else bc_y
    ylo, yhi = (by, by) if isinstance(by, int) else by
    p.bc_lo[0], p.bc_hi[0], p.bc_lo[1], p.bc_hi[1] = lo, hi, ylo, yhi
    p.mode = mode
    p.launch = launch
    p.gravity = gravity
    return p


def grid_1d(n, lo, hi) -> WtGrid:
    g = WtGrid()
    g.ndim = 1
    g.n[0], g.n[1] = n, 1
    g.lo[0], g.hi[0] = lo, hi
    g.lo[1], g.hi[1] = 0.0, 1.0
    return g


def grid_2d(nx, ny, lo=(0.0, 0.0), hi=(1.0, 1.0)) -> WtGrid:
    g = WtGrid()
    g.ndim = 2
    g.n[0], g.n[1] = nx, ny
    g.lo[0], g.lo[1] = lo
    g.hi[0], g.hi[1] = hi
    return g


def _ptr(x):
    """(address, stream) of a torch tensor or numpy array; contiguity and dtype checked."""
    if x is None:
        return None, None
    mod = type(x).__module__
    if mod.startswith("torch"):
        import torch

        if x.dtype not in (torch.float64, torch.uint8, torch.int32, torch.int64):
            raise TypeError("tensor must be float64")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        stream = torch.cuda.current_stream(x.device).cuda_stream if x.is_cuda else None
        return x.data_ptr(), stream
    import numpy as np

    if not isinstance(x, np.ndarray) or not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be a C-contiguous numpy array")
    return x.ctypes.data, None


def _stream(explicit, *arrays):
    if explicit is not None:
        return explicit
    for a in arrays:
        if a is not None:
            s = _ptr(a)[1]
            if s is not None:
                return s
    return None


def workspace_bytes(prob: WtProblem, grid: WtGrid | None, batch_cells=0, nprob=0) -> int:
    n = lib().wt_workspace_bytes(ctypes.byref(prob), ctypes.byref(grid) if grid is not None else None, batch_cells,
                                 nprob)
    if n == 0:
        raise WenoThetaError(WT_ERR_ARG, last_error())
    return n


def adjoint_workspace_bytes(prob, grid, nprob, n_steps, checkpoint_every) -> int:
    n = lib().wt_adjoint_workspace_bytes(ctypes.byref(prob), ctypes.byref(grid), nprob, n_steps, checkpoint_every)
    if n == 0:
        raise WenoThetaError(WT_ERR_ARG, last_error())
    return n


def weno_theta_rhs(prob, grid, u, L, ws, stream=None):
    up, _ = _ptr(u)
    Lp, _ = _ptr(L)
    wp, _ = _ptr(ws)
    _check(lib().weno_theta_rhs(ctypes.byref(prob), ctypes.byref(grid), up, Lp, wp, _nbytes(ws),
                                _stream(stream, u, ws)))


def weno_theta_rhs_noalloc(prob, grid, u, L, stream=None):
    """L(u) with the library's built-in scratch array instead of a caller workspace
    (for callers that cannot allocate device memory); u and L are device arrays."""
    _check(lib().weno_theta_rhs_noalloc(ctypes.byref(prob), ctypes.byref(grid), _ptr(u)[0], _ptr(L)[0],
                                        _stream(stream, u, L)))


def weno_theta_step(prob, grid, u, cfl, ws, dt_fixed=0.0, t_final=float("inf"), max_steps=2**62, stream=None):
    """Integrates u in place; returns (t_reached, steps)."""
    up, _ = _ptr(u)
    wp, _ = _ptr(ws)
    t = ctypes.c_double()
    s = ctypes.c_int64()
    _check(lib().weno_theta_step(ctypes.byref(prob), ctypes.byref(grid), up, cfl, dt_fixed, t_final, max_steps,
                                 ctypes.byref(t), ctypes.byref(s), wp, _nbytes(ws), _stream(stream, u, ws)))
    return t.value, s.value


def weno_theta_step_batched(prob, segs, u_packed, total, cfl, n_steps, ws, t_per_problem=None, stream=None,
                            status_per_problem=None):
    """n_steps RK3 steps of independent 1D problems; ``status_per_problem`` (int32, host or device,
    optional) receives each problem's wt_status, and then a failed problem does not fail the call."""
    arr = (WtSegment * len(segs))(*segs)
    up, _ = _ptr(u_packed)
    tp, _ = _ptr(t_per_problem)
    sp, _ = _ptr(status_per_problem)
    wp, _ = _ptr(ws)
    _check(lib().weno_theta_step_batched(ctypes.byref(prob), arr, len(segs), up, total, cfl, n_steps, tp, sp, wp,
                                         _nbytes(ws), _stream(stream, u_packed, ws)))


def weno_theta_adjoint(prob, grid, nprob, u0, cfl, n_steps, checkpoint_every, dJ_duT, dJ_du0, ws, uT=None,
                       stream=None):
    """Gradient dJ/du0 through n_steps RK3 steps of nprob problems ([nprob][3][n] arrays)."""
    _check(lib().weno_theta_adjoint(ctypes.byref(prob), ctypes.byref(grid), nprob, _ptr(u0)[0], cfl, n_steps,
                                    checkpoint_every, _ptr(dJ_duT)[0], _ptr(dJ_du0)[0], _ptr(uT)[0], _ptr(ws)[0],
                                    _nbytes(ws), _stream(stream, u0, ws)))


def _nbytes(x):
    if type(x).__module__.startswith("torch"):
        return x.numel() * x.element_size()
    return x.nbytes


def alloc_workspace(nbytes, device="cuda"):
    """A device byte buffer of at least nbytes (torch allocations are 512-byte aligned)."""
    import torch

    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def selftest_wait(which, limit_cycles, ws, stream=None):
    """Runs one bounded device-side wait that cannot (which 0, 1, 3, 4) or can (which 2, 5)
    be satisfied (0 grid counter, 1 mbarrier, 3 halo mailbox, 4 and 5 alpha mailbox); returns
    the status (WT_ERR_TIMEOUT when the wait gave up, WT_OK)."""
    wp, _ = _ptr(ws)
    return lib().wt_selftest_wait(which, limit_cycles, wp, _nbytes(ws), _stream(stream, None, ws))

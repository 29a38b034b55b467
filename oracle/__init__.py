"""Plain serial FP64 oracle for the adaptive WENO-theta scheme (arXiv 1504.00731).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
never calls it and shares no code with it.

The arithmetic lives in ``weno_theta_oracle.cpp`` (built here with g++ at
``-O2 -ffp-contract=off``); this module only compiles it and marshals numpy
arrays through ctypes.  Arrays are component-major: ``(m, n)`` in 1D and
``(m, ny, nx)`` in 2D, x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "weno_theta_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libweno_theta_oracle.so")
_lock = threading.Lock()
_lib = None

FLUX_ADVECTION, FLUX_BURGERS, FLUX_EULER1D, FLUX_EULER2D = 0, 1, 2, 3
BC_PERIODIC, BC_OUTFLOW, BC_REFLECTIVE = 0, 1, 2
_M = {FLUX_ADVECTION: 1, FLUX_BURGERS: 1, FLUX_EULER1D: 3, FLUX_EULER2D: 4}


class Problem(ctypes.Structure):
    _fields_ = [
        ("flux", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("adv_speed", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("alpha_R", ctypes.c_double),
        ("bc_lo", ctypes.c_int32 * 2),
        ("bc_hi", ctypes.c_int32 * 2),
        ("gravity", ctypes.c_double),
    ]


def problem(flux, gamma=1.4, adv_speed=1.0, eps=1e-10, alpha_R=50.0, bc=BC_PERIODIC, bc_y=None, gravity=0.0):
    """Build a Problem; ``bc`` is one code or a (lo, hi) pair, ``bc_y`` likewise for 2D; ``gravity``
    is g of the 2D source terms (TEST 6, Sec. 4.3), 0 for none."""
    p = Problem()
    p.flux = flux
    p.m = _M[flux]
    p.gamma = gamma
    p.adv_speed = adv_speed
    p.eps = eps
    p.alpha_R = alpha_R
    lo, hi = (bc, bc) if isinstance(bc, int) else bc
    by = bc if bc_y is None else bc_y
    ylo, yhi = (by, by) if isinstance(by, int) else by
    p.bc_lo[0], p.bc_hi[0] = lo, hi
    p.bc_lo[1], p.bc_hi[1] = ylo, yhi
    p.gravity = gravity
    return p


_BUILD_NOTE = {}


def _compile(out: str, defines=()) -> None:
    """g++ -O2 -ffp-contract=off, with OpenMP over independent problems (and 2D rows and columns)
    where the compiler has it; the arithmetic of each problem, row and column is the same either
    way, so a build without OpenMP gives the same results on one thread."""
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    base = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared"] + [f"-D{d}" for d in defines]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC], capture_output=True, text=True)
    if r.returncode != 0:
        _BUILD_NOTE[out] = "built without OpenMP: " + (r.stderr.strip().splitlines() or ["?"])[-1]
        subprocess.run(base + ["-o", tmp, _SRC], check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (host compiler only) and return its path."""
    with _lock:
        fresh = os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
        if fresh and not force:
            return _SO
        _compile(_SO)
        return _SO


def _load(path, rebuild):
    try:
        return ctypes.CDLL(path)
    except OSError:  # stale library from another architecture
        rebuild()
        return ctypes.CDLL(path)


def planted(name: str):
    """The oracle built with one deliberately wrong line (``-DWTO_PLANT_<name>``), for tests that
    show a pin fails when the oracle is wrong.  Use it with ``using(...)``."""
    path = os.path.join(_BUILD, f"libweno_theta_oracle_plant_{name.lower()}.so")
    with _lock:
        if not (os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            _compile(path, (f"WTO_PLANT_{name}",))
    L = _declare(_load(path, lambda: _compile(path, (f"WTO_PLANT_{name}",))))
    L.wto_set_threads(host_threads())
    return L


class using:
    """Context manager: the module's functions call ``library`` instead of the oracle."""

    def __init__(self, library):
        self.library = library

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = self.library
        return self.library

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def lib():
    """The oracle library, set to use every host core this process may run on (an
    OMP_NUM_THREADS in the environment does not apply: the oracle's threads only split
    independent problems, rows and columns)."""
    global _lib
    if _lib is not None:
        return _lib
    L = _declare(_load(build(), lambda: build(force=True)))
    L.wto_set_threads(host_threads())
    _lib = L
    return _lib


def openmp() -> bool:
    """Whether the oracle library was built with OpenMP."""
    return bool(lib().wto_set_threads(0))


def _declare(L):
    D = ctypes.c_double
    P = ctypes.POINTER(ctypes.c_double)
    I64 = ctypes.c_int64
    PI64 = ctypes.POINTER(ctypes.c_int64)
    PI32 = ctypes.POINTER(ctypes.c_int32)
    PP = ctypes.POINTER(Problem)
    L.wto_weno_theta.argtypes = [P, D, D, PI32, PI32]
    L.wto_weno_theta.restype = D
    L.wto_indicators.argtypes = [P, P]
    L.wto_roe_eigen.argtypes = [ctypes.c_int32, P, P, D, ctypes.c_int32, P, P]
    L.wto_alpha.argtypes = [PP, I64, I64, D, D, P, D, P, P]
    L.wto_rhs.argtypes = [PP, I64, I64, D, D, P, P, PI64, PI64]
    L.wto_rhs_at.argtypes = [PP, I64, I64, D, D, P, P, PI64, I64, P]
    L.wto_rhs_jvp.argtypes = [PP, I64, I64, D, D, P, P, P, P]
    L.wto_run.argtypes = [PP, I64, I64, D, D, P, D, D, D, I64, P, PI64]
    L.wto_run_jvp.argtypes = [PP, I64, I64, D, D, P, P, D, D, D, I64, P, PI64]
    L.wto_count_rhs_ops.argtypes = [PP, I64, I64, D, D, P, PI64]
    L.wto_count_run_ops.argtypes = [PP, I64, I64, D, D, P, D, I64, PI64]
    L.wto_riemann_star.argtypes = [D, D, D, D, D, D, D, P, P, PI32]
    L.wto_riemann_sample.argtypes = [D, D, D, D, D, D, D, D, D, P, I64, P, P, P]
    L.wto_run_batch.argtypes = [PP, ctypes.c_int32, PI64, PI64, P, P, PI32, P, I64, D, I64, ctypes.c_int32, PI64]
    L.wto_run_jvp_batch.argtypes = [PP, ctypes.c_int32, PI64, PI64, P, P, PI32, P, P, I64, D, I64, ctypes.c_int32]
    L.wto_max_threads.restype = ctypes.c_int32
    L.wto_set_threads.argtypes = [ctypes.c_int32]
    L.wto_set_threads.restype = ctypes.c_int32
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    if u.ndim == 2:
        return u, u.shape[1], 1
    if u.ndim == 3:
        return u, u.shape[2], u.shape[1]
    raise ValueError("u must be (m, n) or (m, ny, nx)")


def weno_theta(q, eps=1e-10, alpha_R=50.0):
    """One reconstruction from six split-flux values; returns (value, theta, restricted)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.shape == (6,)
    th = ctypes.c_int32()
    rs = ctypes.c_int32()
    v = lib().wto_weno_theta(_ptr(q), eps, alpha_R, ctypes.byref(th), ctypes.byref(rs))
    return v, th.value, rs.value


def indicators(q):
    """(beta0, beta1, beta2, beta3, tau5, tau6) of one stencil, before the restriction of Eq. (be_res)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(6)
    lib().wto_indicators(_ptr(q), _ptr(out))
    return out


def roe_eigen(Ua, Ub, gamma=1.4, direction=0):
    Ua = np.ascontiguousarray(Ua, dtype=np.float64)
    Ub = np.ascontiguousarray(Ub, dtype=np.float64)
    m = Ua.shape[0]
    R = np.zeros((m, m))
    Lm = np.zeros((m, m))
    lib().wto_roe_eigen(m, _ptr(Ua), _ptr(Ub), gamma, direction, _ptr(R), _ptr(Lm))
    return R, Lm


def alpha(prob, u, dx, dy=1.0, cfl=0.5):
    """Global Lax-Friedrichs constants alpha[dir, s] and the CFL step."""
    u, nx, ny = _dims(u)
    a = np.zeros(8)
    dt = ctypes.c_double()
    lib().wto_alpha(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), cfl, _ptr(a), ctypes.byref(dt))
    return a.reshape(2, 4), dt.value


def rhs(prob, u, dx, dy=1.0, counts=False):
    """L(u) of Eq. (mod_semi); with counts=True also (#theta=1, #restricted) reconstructions."""
    u, nx, ny = _dims(u)
    out = np.zeros_like(u)
    t1 = ctypes.c_int64()
    rs = ctypes.c_int64()
    lib().wto_rhs(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), _ptr(out), ctypes.byref(t1), ctypes.byref(rs))
    if counts:
        return out, t1.value, rs.value
    return out


def rhs_at(prob, u, cells, dx, dy=1.0, alpha8=None):
    """L(u) at flat cell indices (y * nx + x) only; alpha8 defaults to the state's own alphas."""
    u, nx, ny = _dims(u)
    if alpha8 is None:
        alpha8, _ = alpha(prob, u, dx, dy)
    a = np.ascontiguousarray(alpha8, dtype=np.float64).reshape(8)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((cells.size, u.shape[0]))
    lib().wto_rhs_at(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), _ptr(a),
                     cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cells.size, _ptr(out))
    return out


def rhs_jvp(prob, u, du, dx, dy=1.0):
    u, nx, ny = _dims(u)
    du = np.ascontiguousarray(du, dtype=np.float64)
    L = np.zeros_like(u)
    dL = np.zeros_like(u)
    lib().wto_rhs_jvp(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), _ptr(du), _ptr(L), _ptr(dL))
    return L, dL


def run(prob, u, dx, dy=1.0, cfl=0.5, dt_fixed=0.0, t_final=np.inf, n_steps=2**62):
    """TVD-RK3 time integration (Eq. (3rd_RK)); returns (u_final, t, steps)."""
    u, nx, ny = _dims(u)
    u = u.copy()
    t = ctypes.c_double()
    s = ctypes.c_int64()
    lib().wto_run(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), cfl, dt_fixed, t_final, n_steps, ctypes.byref(t),
                  ctypes.byref(s))
    return u, t.value, s.value


def run_jvp(prob, u, du, dx, dy=1.0, cfl=0.5, dt_fixed=0.0, t_final=np.inf, n_steps=2**62):
    """Forward-mode derivative of the run: returns (u_final, du_final, t, steps)."""
    u, nx, ny = _dims(u)
    u = u.copy()
    du = np.ascontiguousarray(du, dtype=np.float64).copy()
    t = ctypes.c_double()
    s = ctypes.c_int64()
    lib().wto_run_jvp(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), _ptr(du), cfl, dt_fixed, t_final, n_steps,
                      ctypes.byref(t), ctypes.byref(s))
    return u, du, t.value, s.value


def count_rhs_ops(prob, u, dx, dy=1.0):
    """Arithmetic operations of one L(u): dict add/mul/div/sqrt/cmp (add counts subtractions)."""
    u, nx, ny = _dims(u)
    out = np.zeros(5, dtype=np.int64)
    lib().wto_count_rhs_ops(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), (int(x) for x in out)))


def count_run_ops(prob, u, dx, dy=1.0, cfl=0.5, n_steps=1):
    """Arithmetic operations of n_steps RK3 steps, CFL step included (add counts subtractions)."""
    u, nx, ny = _dims(u)
    out = np.zeros(5, dtype=np.int64)
    lib().wto_count_run_ops(ctypes.byref(prob), nx, ny, dx, dy, _ptr(u), cfl, n_steps,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), (int(x) for x in out)))


def riemann_star(left, right, gamma=1.4):
    """Star-region (p*, u*, newton iterations) of the exact Riemann problem; states are (rho, u, p)."""
    ps = ctypes.c_double()
    us = ctypes.c_double()
    it = ctypes.c_int32()
    lib().wto_riemann_star(*left, *right, gamma, ctypes.byref(ps), ctypes.byref(us), ctypes.byref(it))
    return ps.value, us.value, it.value


def riemann_sample(left, right, x, x0, t, gamma=1.4):
    """Exact Riemann solution (rho, u, p) at points x and time t, jump at x0."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    rho = np.zeros_like(x)
    u = np.zeros_like(x)
    p = np.zeros_like(x)
    lib().wto_riemann_sample(*left, *right, gamma, x0, t, _ptr(x), x.size, _ptr(rho), _ptr(u), _ptr(p))
    return rho, u, p


def max_threads():
    """Threads ``run_batch`` uses with ``threads=0`` (1 when built without OpenMP)."""
    return int(lib().wto_max_threads())


def run_batch(prob, u_packed, offsets, lengths, lo, hi, bc, cfl=0.5, n_steps=1, threads=0):
    """``n_steps`` TVD-RK3 steps of independent 1D problems in packed planes ``(m, total)``
    (problem p at columns ``offsets[p] .. offsets[p] + lengths[p]``, grid ``[lo[p], hi[p]]``,
    boundary ``bc[p]`` at both ends); each problem is ``run`` on its own, several at once on
    ``threads`` threads (0: all).  Returns (u_packed_final, steps per problem)."""
    u = np.ascontiguousarray(u_packed, dtype=np.float64).copy()
    m, total = u.shape
    nprob = len(lengths)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ln = np.ascontiguousarray(lengths, dtype=np.int64)
    lo = np.ascontiguousarray(np.broadcast_to(lo, (nprob,)), dtype=np.float64)
    hi = np.ascontiguousarray(np.broadcast_to(hi, (nprob,)), dtype=np.float64)
    bc = np.ascontiguousarray(bc, dtype=np.int32)
    steps = np.zeros(nprob, dtype=np.int64)
    I64P = ctypes.POINTER(ctypes.c_int64)
    lib().wto_run_batch(ctypes.byref(prob), nprob, off.ctypes.data_as(I64P), ln.ctypes.data_as(I64P), _ptr(lo),
                        _ptr(hi), bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(u), total, cfl, n_steps,
                        threads, steps.ctypes.data_as(I64P))
    return u, steps


def run_jvp_batch(prob, u_packed, du_packed, offsets, lengths, lo, hi, bc, cfl=0.5, n_steps=1, threads=0):
    """Forward-mode derivative of ``run_batch`` along ``du_packed``: returns (u(T), du(T)), packed
    like the input; each problem is ``run_jvp``'s map, several at once on ``threads`` threads."""
    u = np.ascontiguousarray(u_packed, dtype=np.float64).copy()
    du = np.ascontiguousarray(du_packed, dtype=np.float64).copy()
    m, total = u.shape
    nprob = len(lengths)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ln = np.ascontiguousarray(lengths, dtype=np.int64)
    lo = np.ascontiguousarray(np.broadcast_to(lo, (nprob,)), dtype=np.float64)
    hi = np.ascontiguousarray(np.broadcast_to(hi, (nprob,)), dtype=np.float64)
    bc = np.ascontiguousarray(bc, dtype=np.int32)
    I64P = ctypes.POINTER(ctypes.c_int64)
    lib().wto_run_jvp_batch(ctypes.byref(prob), nprob, off.ctypes.data_as(I64P), ln.ctypes.data_as(I64P), _ptr(lo),
                            _ptr(hi), bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(u), _ptr(du), total,
                            cfl, n_steps, threads)
    return u, du

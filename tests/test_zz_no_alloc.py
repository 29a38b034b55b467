"""weno_theta_rhs_noalloc: the RHS for callers that cannot allocate device memory.

Such callers (a host program with no device allocator, a plug-in held to its host
application's memory budget, a real-time loop where an allocation would synchronise the
device) cannot pass a workspace.  The entry point keeps its scratch in a fixed array built
into the library instead.  It launches the same kernels on the same arguments as
weno_theta_rhs, so its output must be bit for bit the same.  This file is collected last so
that a failure here cannot stop the rest of the suite; it passes alone and after the other
tests, because each call clears what it needs and the array's leftover contents do not
matter.
"""
import ctypes

import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_CELLS = {3: 349498, 1: 1048506}  # the largest n whose padded planes fit the 8 MiB array


def _rhs_with_workspace(b, prob, g, u):
    ws = b.alloc_workspace(b.workspace_bytes(prob, g))
    L = torch.full_like(u, np.nan)
    b.weno_theta_rhs(prob, g, u, L, ws)
    torch.cuda.synchronize()
    return L


def _calls(b):
    rng = np.random.default_rng(21)
    x, dx = W.grid_1d(501, 0.0, 1.0, periodic=False)
    wall = W.cons_1d(0.5 + rng.uniform(size=501), rng.uniform(-1, 1, 501), 0.5 + rng.uniform(size=501))
    return [
        (b.WT_FLUX_EULER1D, b.WT_BC_OUTFLOW, W.euler_c2(4096, seed=11)[0], -5.0, 5.0),
        (b.WT_FLUX_EULER1D, b.WT_BC_PERIODIC, W.euler_riemann(777, W.riemann_params(12), periodic=True)[0],
         -5.0, 5.0),
        (b.WT_FLUX_EULER1D, b.WT_BC_REFLECTIVE, wall, 0.0, 1.0),
        (b.WT_FLUX_ADVECTION, b.WT_BC_PERIODIC, W.advection_ic2(300, 2)[0], -1.0, 1.0),
        (b.WT_FLUX_BURGERS, b.WT_BC_OUTFLOW, W.burgers_sine(333)[0], -1.0, 1.0),
    ]


@pytest.mark.parametrize("mode", [0, 1], ids=["fast", "strict"])
def test_noalloc_rhs_equals_workspace_rhs_on_two_calls(wtlib, mode):
    b = wtlib
    for flux, bc, U, lo, hi in _calls(b):
        prob = b.problem(flux, bc=bc, mode=mode, alpha_R=10.0)
        g = b.grid_1d(U.shape[1], lo, hi)
        u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        ref = _rhs_with_workspace(b, prob, g, u)
        for _ in range(2):  # two calls in a row share the scratch array
            L = torch.full_like(u, np.nan)
            b.weno_theta_rhs_noalloc(prob, g, u, L)
            torch.cuda.synchronize()
            assert torch.equal(L, ref), (flux, bc)


def test_noalloc_strict_rhs_equals_the_oracle(wtlib, oracle):
    b, O = wtlib, oracle
    U, x, dx = W.euler_c2(300, seed=2)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, mode=b.WT_MODE_STRICT, alpha_R=10.0)
    u = torch.from_numpy(U).cuda()
    L = torch.full_like(u, np.nan)
    b.weno_theta_rhs_noalloc(prob, b.grid_1d(300, -5.0, 5.0), u, L)
    torch.cuda.synchronize()
    ref = O.rhs(O.problem(O.FLUX_EULER1D, bc=O.BC_OUTFLOW, alpha_R=10.0), U, dx)
    assert np.array_equal(L.cpu().numpy(), ref)


@pytest.mark.parametrize("m", [3, 1], ids=["euler", "scalar"])
def test_noalloc_at_its_largest_size(wtlib, m):
    """n at the limit fills the array exactly (m padded planes after the control block); the
    result still equals the workspace RHS bit for bit, twice."""
    b = wtlib
    n = MAX_CELLS[m]
    if m == 3:
        U = W.euler_c2(n, seed=5)[0]
        prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, alpha_R=10.0)
    else:
        U = W.advection_seeded(n, seed=5)[0]
        prob = b.problem(b.WT_FLUX_ADVECTION, bc=b.WT_BC_PERIODIC)
    g = b.grid_1d(n, -5.0, 5.0)
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    ref = _rhs_with_workspace(b, prob, g, u)
    for _ in range(2):
        L = torch.full_like(u, np.nan)
        b.weno_theta_rhs_noalloc(prob, g, u, L)
        torch.cuda.synchronize()
        assert torch.equal(L, ref)


@pytest.mark.parametrize("m", [3, 1], ids=["euler", "scalar"])
def test_noalloc_rejects_sizes_beyond_its_scratch(wtlib, m):
    b = wtlib
    prob = b.problem(b.WT_FLUX_EULER1D if m == 3 else b.WT_FLUX_ADVECTION, bc=b.WT_BC_OUTFLOW)
    n = MAX_CELLS[m] + 1
    g = b.grid_1d(n, -5.0, 5.0)
    u = torch.ones((m, n), dtype=torch.float64, device="cuda")
    L = torch.empty_like(u)
    status = b.lib().weno_theta_rhs_noalloc(ctypes.byref(prob), ctypes.byref(g), u.data_ptr(), L.data_ptr(), None)
    assert status == b.WT_ERR_ARG
    assert "scratch" in b.last_error()


def test_noalloc_checks_its_arguments_like_the_workspace_rhs(wtlib):
    """The same argument checks as weno_theta_rhs: a gravity source on a 1D flux is unsupported,
    a non-finite eps or domain and an unknown boundary are rejected."""
    b = wtlib
    g = b.grid_1d(64, -1.0, 1.0)
    u = torch.ones((3, 64), dtype=torch.float64, device="cuda")
    L = torch.empty_like(u)

    def status(prob, grid=g):
        return b.lib().weno_theta_rhs_noalloc(ctypes.byref(prob), ctypes.byref(grid), u.data_ptr(), L.data_ptr(), None)

    assert status(b.problem(b.WT_FLUX_EULER1D, gravity=0.1)) == b.WT_ERR_UNSUPPORTED
    assert status(b.problem(b.WT_FLUX_EULER1D, eps=float("nan"))) == b.WT_ERR_ARG
    bad_bc = b.problem(b.WT_FLUX_EULER1D)
    bad_bc.bc_lo[1] = 7
    assert status(bad_bc) == b.WT_ERR_ARG
    assert status(b.problem(b.WT_FLUX_EULER1D), b.grid_1d(64, 0.0, float("inf"))) == b.WT_ERR_ARG

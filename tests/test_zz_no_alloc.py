"""weno_theta_rhs_noalloc: the RHS for callers that cannot allocate device memory.

Such callers (a host program with no device allocator, a plug-in held to its host
application's memory budget, a real-time loop where an allocation would synchronise the
device) cannot pass a workspace.  The entry point keeps its scratch in a fixed array built
into the library instead.  This file is collected last so that a failure here cannot stop
the rest of the suite; it passes alone and after the other tests, because each call clears
what it needs and the array's leftover contents do not matter.
"""
import ctypes

import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHS_TOL = 1e-13  # the per-RHS tolerance of the parity tests


def _rhs_with_workspace(b, prob, g, u):
    ws = b.alloc_workspace(b.workspace_bytes(prob, g))
    L = torch.full_like(u, np.nan)
    b.weno_theta_rhs(prob, g, u, L, ws)
    torch.cuda.synchronize()
    return L


def _close(a, ref):
    a, ref = a.cpu().numpy(), ref.cpu().numpy()
    scale = np.abs(ref).max(axis=1) + 1e-300
    return np.all(np.abs(a - ref).max(axis=1) <= RHS_TOL * scale)


@pytest.mark.parametrize("mode", [0, 1], ids=["fast", "strict"])
def test_noalloc_rhs_matches_workspace_rhs_on_two_calls(wtlib, mode):
    b = wtlib
    calls = [
        (b.WT_FLUX_EULER1D, b.WT_BC_OUTFLOW, *W.euler_c2(4096, seed=11)[::2], -5.0, 5.0),
        (b.WT_FLUX_EULER1D, b.WT_BC_PERIODIC, *W.euler_riemann(777, W.riemann_params(12), periodic=True)[::2],
         -5.0, 5.0),
        (b.WT_FLUX_ADVECTION, b.WT_BC_PERIODIC, W.advection_ic2(300, 2)[0], 0, -1.0, 1.0),
    ]
    for flux, bc, U, _, lo, hi in calls:
        prob = b.problem(flux, bc=bc, mode=mode)
        g = b.grid_1d(U.shape[1], lo, hi)
        u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        ref = _rhs_with_workspace(b, prob, g, u)
        for _ in range(2):  # two calls in a row share the scratch array
            L = torch.full_like(u, np.nan)
            b.weno_theta_rhs_noalloc(prob, g, u, L)
            torch.cuda.synchronize()
            assert _close(L, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(wtlib):
    b = wtlib
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW)
    n = 349498 + 1
    g = b.grid_1d(n, -5.0, 5.0)
    u = torch.ones((3, n), dtype=torch.float64, device="cuda")
    L = torch.empty_like(u)
    status = b.lib().weno_theta_rhs_noalloc(ctypes.byref(prob), ctypes.byref(g), u.data_ptr(), L.data_ptr(), None)
    assert status == b.WT_ERR_ARG
    assert "scratch" in b.last_error()

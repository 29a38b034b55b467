"""The C ABI library loads, exports every entry point include/weno_theta.h declares, and
rejects bad arguments on the host before touching a GPU (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "weno_theta.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:int|size_t|const char\*)\s+(\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("weno_theta_rhs", "weno_theta_step", "weno_theta_step_batched", "weno_theta_adjoint",
                     "wt_workspace_bytes", "wt_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(wtlib):
    L = wtlib.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(wtlib.EXPORTED)


def test_struct_layouts_match_header(wtlib):
    # wt_problem: 2 int32, 4 doubles, 4 int32 bc, mode, reserved
    assert ctypes.sizeof(wtlib.WtProblem) == 4 + 4 + 8 * 4 + 4 * 4 + 4 + 4
    assert wtlib.WtProblem.gamma.offset == 8
    assert wtlib.WtProblem.bc_lo.offset == 40
    assert ctypes.sizeof(wtlib.WtGrid) == 4 + 4 + 16 + 16 + 16
    assert ctypes.sizeof(wtlib.WtSegment) == 8 + 8 + 8 + 8 + 4 + 4


def test_workspace_size_and_argument_checks(wtlib):
    b = wtlib
    p = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW)
    g = b.grid_1d(4096, -5.0, 5.0)
    n = b.workspace_bytes(p, g)
    assert n >= 3 * 3 * 4102 * 8 and n % 256 == 0
    bad = b.problem(b.WT_FLUX_EULER1D)
    bad.m = 4
    with pytest.raises(b.WenoThetaError) as e:
        b.workspace_bytes(bad, g)
    assert "m = 4" in b.last_error()
    g2 = b.grid_1d(2, -1.0, 1.0)
    with pytest.raises(b.WenoThetaError):
        b.workspace_bytes(p, g2)
    # host-side rejection before any CUDA call: NULL problem, NULL workspace
    L = b.lib()
    u = np.zeros((3, 16))
    assert L.weno_theta_rhs(None, ctypes.byref(g), u.ctypes.data, u.ctypes.data, None, 0, None) == b.WT_ERR_ARG
    g16 = b.grid_1d(16, 0.0, 1.0)
    assert L.weno_theta_rhs(ctypes.byref(p), ctypes.byref(g16), u.ctypes.data, u.ctypes.data, None, 0,
                            None) == b.WT_ERR_WORKSPACE
    sc = b.problem(b.WT_FLUX_ADVECTION, bc=b.WT_BC_REFLECTIVE)
    assert L.weno_theta_rhs(ctypes.byref(sc), ctypes.byref(g16), u.ctypes.data, u.ctypes.data, None, 0,
                            None) == b.WT_ERR_UNSUPPORTED
    mixed = b.problem(b.WT_FLUX_EULER1D, bc=(b.WT_BC_PERIODIC, b.WT_BC_OUTFLOW))
    assert L.weno_theta_rhs(ctypes.byref(mixed), ctypes.byref(g16), u.ctypes.data, u.ctypes.data, None, 0,
                            None) == b.WT_ERR_ARG

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


def test_struct_layouts_match_header(wtlib, tmp_path):
    """The ctypes mirrors of the public structs against the C compiler's view of the header."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    fields = {"wt_problem": ("flux", "m", "gamma", "adv_speed", "eps", "alpha_R", "bc_lo", "bc_hi", "mode",
                             "launch", "gravity"),
              "wt_grid": ("ndim", "reserved", "n", "lo", "hi"),
              "wt_segment": ("offset", "n", "lo", "hi", "bc_lo", "bc_hi")}
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include <cuda_runtime_api.h>", '#include "weno_theta.h"',
             "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    r = subprocess.run(["gcc", "-I", inc, "-I", cuda_inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("header needs the CUDA runtime headers: " + r.stderr[:200])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        st, f, v = line.split()
        got[(st, f)] = int(v)
    for st, cls in (("wt_problem", wtlib.WtProblem), ("wt_grid", wtlib.WtGrid), ("wt_segment", wtlib.WtSegment)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)


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


def test_gravity_is_checked_on_the_host(wtlib):
    """Gravity source terms belong to the 2D Euler equations (TEST 6, Sec. 4.3): a nonzero g for
    another flux is unsupported, a non-finite g is an argument error."""
    b = wtlib
    L = b.lib()
    u = np.zeros((3, 16))
    g16 = b.grid_1d(16, 0.0, 1.0)
    grav1d = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, gravity=0.1)
    assert L.weno_theta_rhs(ctypes.byref(grav1d), ctypes.byref(g16), u.ctypes.data, u.ctypes.data, None, 0,
                            None) == b.WT_ERR_UNSUPPORTED
    nan = b.problem(b.WT_FLUX_EULER2D, bc=b.WT_BC_PERIODIC, gravity=float("nan"))
    g2 = b.grid_2d(8, 8)
    u2 = np.zeros((4, 8, 8))
    assert L.weno_theta_rhs(ctypes.byref(nan), ctypes.byref(g2), u2.ctypes.data, u2.ctypes.data, None, 0,
                            None) == b.WT_ERR_ARG
    ok = b.problem(b.WT_FLUX_EULER2D, bc=b.WT_BC_PERIODIC, bc_y=b.WT_BC_REFLECTIVE, gravity=0.1)
    assert b.workspace_bytes(ok, g2) > 0


def test_selftest_wait_checks_arguments_on_the_host(wtlib):
    b = wtlib
    L = b.lib()
    assert L.wt_selftest_wait(7, 1000, None, 0, None) == b.WT_ERR_ARG
    assert L.wt_selftest_wait(0, 0, None, 0, None) == b.WT_ERR_ARG
    assert L.wt_selftest_wait(0, 1 << 40, None, 0, None) == b.WT_ERR_ARG
    assert L.wt_selftest_wait(0, 1000, None, 0, None) == b.WT_ERR_WORKSPACE

"""GPU path (through the C ABI) against the CPU oracle on the same seeded inputs.

Strict mode evaluates the paper's formulas literally and must match the oracle bit for
bit, per RHS evaluation and after whole runs.  Fast mode must match within the stated
tolerances: 1e-13 per RHS evaluation, normwise per component,
max_j |L_gpu - L_oracle| <= 1e-13 max_j |L_oracle|; and at final time 1e-10 in L_inf on
smooth runs and 1e-10 in L1 (dx * sum |du|) on shock runs.
"""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHS_TOL = 1e-13
SMOOTH_LINF_TOL = 1e-10
SHOCK_L1_TOL = 1e-10


def _oracle_problem(O, b, prob):
    return O.problem(prob.flux, gamma=prob.gamma, adv_speed=prob.adv_speed, eps=prob.eps, alpha_R=prob.alpha_R,
                     bc=(prob.bc_lo[0], prob.bc_hi[0]))


def _gpu_rhs(b, prob, U, lo, hi):
    n = U.shape[1]
    g = b.grid_1d(n, lo, hi)
    ws = b.alloc_workspace(b.workspace_bytes(prob, g))
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    L = torch.full_like(u, np.nan)
    b.weno_theta_rhs(prob, g, u, L, ws)
    torch.cuda.synchronize()
    return L.cpu().numpy()


def _gpu_run(b, prob, U, lo, hi, **kw):
    n = U.shape[1]
    g = b.grid_1d(n, lo, hi)
    ws = b.alloc_workspace(b.workspace_bytes(prob, g))
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    t, steps = b.weno_theta_step(prob, g, u, ws=ws, **kw)
    return u.cpu().numpy(), t, steps


def _cases():
    """(name, flux, bc, U, lo, hi) on seeded inputs, several tiles and ragged tails."""
    out = []
    u, x, dx = W.advection_sine(200)
    out.append(("adv-sine-200", 0, 0, u, -1.0, 1.0))
    u, x, dx, _ = W.advection_seeded(257, 7)
    out.append(("adv-seeded-257", 0, 0, u, -1.0, 1.0))
    for n in (3, 5, 64, 128, 129, 300):
        u, _, _ = W.advection_ic2(n, 2)
        out.append((f"adv-ic2-{n}", 0, 0, u, -1.0, 1.0))
    xb, _ = W.grid_1d(100, -1.0, 1.0, periodic=False)
    out.append(("burgers-100", 1, 1, (np.sin(np.pi * xb) + 0.5 * (xb > 0.2))[None, :], -1.0, 1.0))
    for n in (3, 4, 31, 32, 62, 63, 64, 126, 127, 128, 129, 500, 4096):
        U, _, _ = W.euler_riemann(n, W.riemann_params(n))
        out.append((f"euler-outflow-{n}", 2, 1, U, -5.0, 5.0))
    U, _, _ = W.euler_riemann(1000, W.riemann_params(3), periodic=True)
    out.append(("euler-periodic-1000", 2, 0, U, -5.0, 5.0))
    U, _, _ = W.symmetric_123(130)
    out.append(("euler-reflective-130", 2, 2, U, -5.0, 5.0))
    U, _, _ = W.sod(300)
    out.append(("euler-sod-300", 2, 1, U, -5.0, 5.0))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_rhs_strict_is_bitwise(wtlib, oracle, case):
    b, O = wtlib, oracle
    name, flux, bc, U, lo, hi = case
    prob = b.problem(flux, bc=bc, mode=b.WT_MODE_STRICT)
    L = _gpu_rhs(b, prob, U, lo, hi)
    ref = O.rhs(_oracle_problem(O, b, prob), U, (hi - lo) / U.shape[1])
    assert np.array_equal(L, ref), np.abs(L - ref).max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_rhs_fast_within_tolerance(wtlib, oracle, case):
    b, O = wtlib, oracle
    name, flux, bc, U, lo, hi = case
    prob = b.problem(flux, bc=bc, mode=b.WT_MODE_FAST)
    L = _gpu_rhs(b, prob, U, lo, hi)
    ref = O.rhs(_oracle_problem(O, b, prob), U, (hi - lo) / U.shape[1])
    scale = np.abs(ref).max(axis=1) + 1e-300
    err = np.abs(L - ref).max(axis=1)
    assert np.all(err <= RHS_TOL * scale), (err / scale)


def test_host_and_device_arrays_agree(wtlib):
    b = wtlib
    U, _, _ = W.euler_c2(777, seed=5)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW)
    L_dev = _gpu_rhs(b, prob, U, -5.0, 5.0)
    g = b.grid_1d(777, -5.0, 5.0)
    ws = b.alloc_workspace(b.workspace_bytes(prob, g))
    L_host = np.zeros_like(U)
    b.weno_theta_rhs(prob, g, np.ascontiguousarray(U), L_host, ws)
    assert np.array_equal(L_dev, L_host)
    u_host = np.ascontiguousarray(U).copy()
    t, s = b.weno_theta_step(prob, g, u_host, 0.5, ws, max_steps=25)
    u_dev, t2, s2 = _gpu_run(b, prob, U, -5.0, 5.0, cfl=0.5, max_steps=25)
    assert s == s2 == 25 and t == t2
    assert np.array_equal(u_host, u_dev)


def test_linear_advection_run_strict_bitwise_and_table1(wtlib, oracle):
    """Config: u_t + u_x = 0 on [-1, 1], periodic, N = 200, CFL 0.4 to t = 2 (500 steps)."""
    b, O = wtlib, oracle
    u0, x, dx = W.advection_sine(200)
    for mode in (b.WT_MODE_STRICT, b.WT_MODE_FAST):
        prob = b.problem(b.WT_FLUX_ADVECTION, mode=mode)
        u, t, steps = _gpu_run(b, prob, u0, -1.0, 1.0, cfl=0.4, t_final=2.0)
        ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), u0, dx, cfl=0.4, t_final=2.0)
        assert t == t_ref == 2.0 and steps == s_ref
        if mode == b.WT_MODE_STRICT:
            assert np.array_equal(u, ref)
        else:
            assert np.abs(u - ref).max() <= SMOOTH_LINF_TOL
    # seeded variant, and the Table 1 setting (dt = dx^2, t = 1) on the GPU
    u0, x, dx, (a, phi) = W.advection_seeded(200, 1)
    prob = b.problem(b.WT_FLUX_ADVECTION)
    u, _, _ = _gpu_run(b, prob, u0, -1.0, 1.0, cfl=0.4, t_final=2.0)
    ref, _, _ = O.run(_oracle_problem(O, b, prob), u0, dx, cfl=0.4, t_final=2.0)
    assert np.abs(u - ref).max() <= SMOOTH_LINF_TOL
    u0, x, dx = W.advection_sine(80)
    u, t, _ = _gpu_run(b, prob, u0, -1.0, 1.0, dt_fixed=dx * dx, cfl=0.4, t_final=1.0)
    assert t == 1.0
    assert abs(np.abs(u[0] - np.sin(np.pi * (x - 1.0))).max() - 5.3e-9) < 0.05e-9  # Table 1, N = 80


def test_euler_run_strict_bitwise(wtlib, oracle):
    b, O = wtlib, oracle
    for n, seed, bc, steps in ((512, 1, 1, 200), (301, 2, 0, 150), (130, 0, 2, 100)):
        periodic = bc == 0
        if bc == 2:
            U, x, dx = W.symmetric_123(n)
        else:
            U, x, dx = W.euler_riemann(n, W.riemann_params(seed), periodic=periodic)
        prob = b.problem(b.WT_FLUX_EULER1D, bc=bc, mode=b.WT_MODE_STRICT)
        u, t, s = _gpu_run(b, prob, U, -5.0, 5.0, cfl=0.5, max_steps=steps)
        ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), U, dx, cfl=0.5, n_steps=steps)
        assert s == s_ref == steps and t == t_ref
        assert np.array_equal(u, ref), np.abs(u - ref).max()


def test_all_launch_strategies_are_bitwise(wtlib, oracle):
    """The step entry point picks its launch by how the grid's tiles fit on the device: the
    step-blocked persistent kernel (at most one tile per SM: up to 4104 Euler / 7752 scalar
    cells), the persistent kernel with a halo exchange per stage (all tiles co-resident), or
    CUDA graphs of the stage kernels.  All three are bitwise equal to the oracle in strict mode."""
    b, O = wtlib, oracle
    cases = ((2, 2000, 1), (2, 4104, 0), (2, 20000, 1), (2, 40000, 1),
             (0, 1000, 0), (0, 10000, 0), (0, 20000, 0), (1, 7000, 1))
    for flux, n, bc in cases:
        steps = 4
        if flux == 2:
            U, x, dx = W.euler_riemann(n, W.riemann_params(n), periodic=bc == 0)
            lo, hi = -5.0, 5.0
        else:
            U, _, _ = W.advection_ic2(n, 2)
            if flux == 1:
                U = U + 0.5
            lo, hi = -1.0, 1.0
            dx = (hi - lo) / n
        prob = b.problem(flux, bc=bc, mode=b.WT_MODE_STRICT)
        u, t, s = _gpu_run(b, prob, U, lo, hi, cfl=0.5, max_steps=steps)
        ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), U, dx, cfl=0.5, n_steps=steps)
        assert s == s_ref == steps and t == t_ref, (flux, n)
        assert np.array_equal(u, ref), (flux, n, np.abs(u - ref).max())


@pytest.mark.parametrize("bc", [0, 1, 2], ids=["periodic", "outflow", "reflective"])
def test_tiny_and_ragged_grids_run_bitwise(wtlib, oracle, bc):
    """Grids shorter than the 9 halo cells a step-blocked tile carries per side, and ragged
    last tiles (1, 2, 8, 9 and 26 cells), for every boundary condition, 6 steps."""
    b, O = wtlib, oracle
    for n in (3, 4, 5, 8, 9, 10, 17, 28, 29, 35, 36, 54, 80):
        U, x, dx = W.euler_riemann(n, W.riemann_params(n + 7), periodic=bc == 0)
        prob = b.problem(b.WT_FLUX_EULER1D, bc=bc, mode=b.WT_MODE_STRICT, alpha_R=W.ALPHA_R_SEEDED)
        ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), U, dx, cfl=0.5, n_steps=6)
        if not np.isfinite(ref).all():
            # the oracle's state blows up too (periodic n = 4): the GPU path must report it
            with pytest.raises(b.WenoThetaError) as e:
                _gpu_run(b, prob, U, -5.0, 5.0, cfl=0.5, max_steps=6)
            assert e.value.status == b.WT_ERR_NONPHYSICAL
            continue
        u, t, s = _gpu_run(b, prob, U, -5.0, 5.0, cfl=0.5, max_steps=6)
        assert s == s_ref == 6 and t == t_ref, n
        assert np.array_equal(u, ref), (n, np.abs(u - ref).max())
        if bc == 2:
            continue  # reflective walls are defined for the Euler equations only
        V, _, _ = W.advection_ic2(n, 2)
        pa = b.problem(b.WT_FLUX_BURGERS, bc=bc, mode=b.WT_MODE_STRICT)
        V = V + 0.3
        u, t, s = _gpu_run(b, pa, V, -1.0, 1.0, cfl=0.5, max_steps=6)
        ref, t_ref, s_ref = O.run(_oracle_problem(O, b, pa), V, 2.0 / n, cfl=0.5, n_steps=6)
        assert s == s_ref == 6 and t == t_ref, n
        assert np.array_equal(u, ref), (n, np.abs(u - ref).max())


def test_persistent_run_across_launch_chunks(wtlib, oracle):
    """More steps than one persistent launch takes (4096): the run resumes across launches
    with the same alpha slots and time, bit for bit."""
    b, O = wtlib, oracle
    U, _, _ = W.advection_ic2(64, 2)
    prob = b.problem(b.WT_FLUX_ADVECTION, bc=b.WT_BC_PERIODIC, mode=b.WT_MODE_STRICT)
    u, t, s = _gpu_run(b, prob, U, -1.0, 1.0, cfl=0.4, max_steps=4100)
    ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), U, 2.0 / 64, cfl=0.4, n_steps=4100)
    assert s == s_ref == 4100 and t == t_ref
    assert np.array_equal(u, ref)


def test_euler_run_to_final_time(wtlib, oracle):
    """t_final-bounded run: the last step is clipped and the run stops exactly at t_final."""
    b, O = wtlib, oracle
    U, x, dx = W.sod(300)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, mode=b.WT_MODE_STRICT)
    u, t, s = _gpu_run(b, prob, U, -5.0, 5.0, cfl=0.5, t_final=1.7)
    ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), U, dx, cfl=0.5, t_final=1.7)
    assert t == t_ref == 1.7 and s == s_ref
    assert np.array_equal(u, ref)


def test_euler_full_size_fast_run(wtlib, oracle):
    """The benchmark configuration, as bench.py launches it: 1D Euler, N = 4096 on [-5, 5],
    outflow, seeded Riemann + entropy-wave data, CFL 0.5, 2000 RK steps, fast mode."""
    b, O = wtlib, oracle
    U, x, dx = W.euler_c2(4096, seed=0)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, alpha_R=W.ALPHA_R_SEEDED)
    u, t, s = _gpu_run(b, prob, U, -5.0, 5.0, cfl=0.5, max_steps=2000)
    ref, t_ref, s_ref = O.run(_oracle_problem(O, b, prob), U, dx, cfl=0.5, n_steps=2000)
    assert s == s_ref == 2000
    assert abs(t - t_ref) <= 1e-12 * t_ref
    l1 = dx * np.abs(u - ref).sum(axis=1)
    assert np.all(l1 <= SHOCK_L1_TOL), l1


def test_nonphysical_state_is_reported_not_hidden(wtlib):
    b = wtlib
    U, _, _ = W.euler_c2(256, seed=3)
    U[0, 100] = -1.0
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW)
    u_in = U.copy()
    g = b.grid_1d(256, -5.0, 5.0)
    ws = b.alloc_workspace(b.workspace_bytes(prob, g))
    u = torch.from_numpy(u_in).cuda()
    with pytest.raises(b.WenoThetaError) as e:
        b.weno_theta_step(prob, g, u, 0.5, ws, max_steps=3)
    assert e.value.status == b.WT_ERR_NONPHYSICAL
    assert np.array_equal(u.cpu().numpy(), U)  # input untouched on error
    # the context is still usable
    U2, _, _ = W.euler_c2(256, seed=3)
    u2 = torch.from_numpy(U2).cuda()
    b.weno_theta_step(prob, g, u2, 0.5, ws, max_steps=3)


@pytest.mark.parametrize("mode", ["strict", "fast"])
def test_launch_strategies_agree_bit_for_bit(wtlib, mode):
    """weno_theta_step through the step-blocked kernel (the automatic choice for these sizes)
    and through per-stage launches of the fused stage kernel give the same state, in either
    arithmetic policy: shock data whose stencils take every path (screened, deferred, weights)."""
    b = wtlib
    md = b.WT_MODE_STRICT if mode == "strict" else b.WT_MODE_FAST
    cases = [(b.WT_FLUX_EULER1D, b.WT_BC_OUTFLOW, W.euler_c2(300, seed=5)[0], -5.0, 5.0),
             (b.WT_FLUX_EULER1D, b.WT_BC_PERIODIC, W.euler_c2(1000, seed=6)[0], -5.0, 5.0),
             (b.WT_FLUX_BURGERS, b.WT_BC_PERIODIC, W.advection_ic2(200, 2)[0] + 0.3, -1.0, 1.0)]
    for flux, bc, U, lo, hi in cases:
        out = []
        for launch in (b.WT_LAUNCH_AUTO, b.WT_LAUNCH_STAGES):
            prob = b.problem(flux, bc=bc, mode=md, alpha_R=W.ALPHA_R_SEEDED, launch=launch)
            n = U.shape[-1]
            g = b.grid_1d(n, lo, hi)
            ws = b.alloc_workspace(b.workspace_bytes(prob, g))
            u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
            t, s = b.weno_theta_step(prob, g, u, 0.5, ws, max_steps=40)
            out.append((u.cpu().numpy(), t, s))
        assert out[0][2] == out[1][2] == 40 and out[0][1] == out[1][1], (flux, bc)
        assert np.array_equal(out[0][0], out[1][0]), (flux, bc, np.abs(out[0][0] - out[1][0]).max())

"""The test problems of Sec. 4.2 / 4.3 that exercise reflective walls and gravity, on the GPU
against the oracle: two interacting blast waves (TEST 5), the Rayleigh-Taylor instability with
its gravity source terms (TEST 6) and the implosion problem (TEST 7).  Strict mode is bitwise
equal to the oracle; fast mode is within the tolerances of the other parity tests.  On the
paper's grids, the symmetry the paper reports for WENO-theta holds to round-off."""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHS_TOL = 1e-13
SHOCK_L1_TOL = 1e-10


def _run(b, prob, U, grid, **kw):
    ws = b.alloc_workspace(b.workspace_bytes(prob, grid))
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    t, s = b.weno_theta_step(prob, grid, u, ws=ws, **kw)
    return u.cpu().numpy(), t, s


def _rhs(b, prob, U, grid):
    ws = b.alloc_workspace(b.workspace_bytes(prob, grid))
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    L = torch.full_like(u, np.nan)
    b.weno_theta_rhs(prob, grid, u, L, ws)
    torch.cuda.synchronize()
    return L.cpu().numpy()


def _rhs_tolerance(U, ref, h):
    """Fast and strict interface fluxes differ by a few ulp of the flux, and L = -dh/dx turns
    that into ~ulp(max |f|) / dx.  Where the RHS is a small difference of large fluxes (the
    hydrostatic pressure of the Rayleigh-Taylor data, L_x of rho u vanishing by symmetry) that
    exceeds 1e-13 of max |L|, so the bound per component is the larger of 1e-13 max |L| and
    50 ulp of the largest physical flux over h."""
    rho, mu, mv, E = U
    u, v = mu / rho, mv / rho
    p = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    fmax = max(np.abs(a).max() for a in (mu, mu * u + p, mu * v, u * (E + p), mv * v + p, v * (E + p)))
    return np.maximum(RHS_TOL * np.abs(ref).reshape(4, -1).max(axis=1), 50 * 2.2e-16 * fmax / h)


def _rt(b, O, nx, ny, mode):
    U, dx, dy = W.rayleigh_taylor(nx, ny)
    gp = b.problem(b.WT_FLUX_EULER2D, bc=b.WT_BC_PERIODIC, bc_y=b.WT_BC_REFLECTIVE, mode=mode, gravity=W.RT_GRAVITY)
    op = O.problem(O.FLUX_EULER2D, bc=O.BC_PERIODIC, bc_y=O.BC_REFLECTIVE, gravity=W.RT_GRAVITY)
    return U, dx, dy, gp, op, b.grid_2d(nx, ny, (-0.25, -0.75), (0.25, 0.75))


def _implosion(b, O, n, mode):
    U, dx, dy = W.implosion(n)
    gp = b.problem(b.WT_FLUX_EULER2D, bc=b.WT_BC_REFLECTIVE, bc_y=b.WT_BC_REFLECTIVE, mode=mode, alpha_R=1.0)
    op = O.problem(O.FLUX_EULER2D, bc=O.BC_REFLECTIVE, bc_y=O.BC_REFLECTIVE, alpha_R=1.0)
    return U, dx, dy, gp, op, b.grid_2d(n, n)


@pytest.mark.parametrize("name", ["rayleigh_taylor", "implosion"])
def test_rhs_and_run_match_the_oracle(wtlib, oracle, name):
    b, O = wtlib, oracle
    make = {"rayleigh_taylor": lambda mode: _rt(b, O, 24, 72, mode),
            "implosion": lambda mode: _implosion(b, O, 40, mode)}[name]
    U, dx, dy, gp, op, grid = make(b.WT_MODE_STRICT)
    ref = O.rhs(op, U, dx, dy)
    assert np.array_equal(_rhs(b, gp, U, grid), ref)
    r_ref, t_ref, s_ref = O.run(op, U, dx, dy, cfl=0.5, n_steps=15)
    u, t, s = _run(b, gp, U, grid, cfl=0.5, max_steps=15)
    assert s == s_ref == 15 and t == t_ref
    assert np.array_equal(u, r_ref), np.abs(u - r_ref).max()
    U, dx, dy, gp, op, grid = make(b.WT_MODE_FAST)
    L = _rhs(b, gp, U, grid)
    err = np.abs(L - ref).reshape(4, -1).max(axis=1)
    assert np.all(err <= _rhs_tolerance(U, ref, min(dx, dy))), err
    u, t, s = _run(b, gp, U, grid, cfl=0.5, max_steps=15)
    l1 = dx * dy * np.abs(u - r_ref).reshape(4, -1).sum(axis=1)
    assert np.all(l1 <= SHOCK_L1_TOL), l1


def test_blast_waves_match_the_oracle(wtlib, oracle):
    """TEST 5 on the paper's grid (N = 801), reflective walls, alpha_R = 10, to t = 0.004 (the
    blasts have left their initial positions and the left fan has hit the wall)."""
    b, O = wtlib, oracle
    U, x, dx = W.blast_waves(801)
    op = O.problem(O.FLUX_EULER1D, bc=O.BC_REFLECTIVE, alpha_R=10.0)
    r_ref, t_ref, s_ref = O.run(op, U, dx, cfl=0.5, t_final=0.004)
    grid = b.grid_1d(801, 0.0, 1.0)
    for mode in (b.WT_MODE_STRICT, b.WT_MODE_FAST):
        gp = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_REFLECTIVE, mode=mode, alpha_R=10.0)
        u, t, s = _run(b, gp, U, grid, cfl=0.5, t_final=0.004)
        if mode == b.WT_MODE_STRICT:
            assert t == t_ref == 0.004 and s == s_ref
            assert np.array_equal(u, r_ref)
        else:
            # 1e-10 in L1, or ten times the oracle's own spread when its data move by one ulp
            spread = np.zeros(3)
            for seed in (1, 2, 3):
                other, _, _ = O.run(op, W.ulp_perturbed(U, seed), dx, cfl=0.5, t_final=0.004)
                spread = np.maximum(spread, dx * np.abs(other - r_ref).sum(axis=1))
            assert abs(t - 0.004) <= 1e-15 and s == s_ref
            l1 = dx * np.abs(u - r_ref).sum(axis=1)
            assert np.all(l1 <= np.maximum(SHOCK_L1_TOL, 10.0 * spread)), (l1, spread)


def _mirror_rt(u):
    return np.stack([sg * u[c][:, ::-1] for c, sg in enumerate((1.0, -1.0, 1.0, 1.0))])


def _transpose(u):
    return np.stack([u[0].T, u[2].T, u[1].T, u[3].T])


def test_rayleigh_taylor_keeps_its_symmetry_on_the_paper_grid(wtlib, oracle):
    """120 x 360, CFL 0.5, to t = 9.5 (the run of the paper's Rayleigh-Taylor figure), fast
    mode: the state stays mirror-symmetric about x = 0 bit for bit while the interface rolls
    up; strict mode likewise to t = 1."""
    b, O = wtlib, oracle
    for mode, tf, grown in ((b.WT_MODE_FAST, 9.5, 1e-3), (b.WT_MODE_STRICT, 1.0, 1e-4)):
        U, dx, dy, gp, op, grid = _rt(b, O, 120, 360, mode)
        u, t, s = _run(b, gp, U, grid, cfl=0.5, t_final=tf)
        assert t == tf and np.isfinite(u).all()
        assert np.abs(u[1]).max() > grown * np.abs(u).max()  # lateral motion has developed
        assert np.array_equal(u, _mirror_rt(u)), (mode, np.abs(u - _mirror_rt(u)).max())


def test_implosion_keeps_its_symmetry_on_the_paper_grid(wtlib, oracle):
    """400 x 400, alpha_R = 1, fast mode to t = 2 and strict mode to t = 0.25: the state is
    symmetric about the diagonal x = y bit for bit."""
    b, O = wtlib, oracle
    for mode, tf in ((b.WT_MODE_FAST, 2.0), (b.WT_MODE_STRICT, 0.25)):
        U, dx, dy, gp, op, grid = _implosion(b, O, 400, mode)
        u, t, s = _run(b, gp, U, grid, cfl=0.5, t_final=tf)
        assert t == tf and np.isfinite(u).all()
        assert np.array_equal(u, _transpose(u)), (mode, np.abs(u - _transpose(u)).max())


VALIDATION = [
    # (name, flux, workload, bc, alpha_R, cfl, t_final, lo, hi)
    ("resolution-max-sin-N200", 0, lambda: W.sine_max(200), 0, 50.0, 0.4, 2.4, -1.0, 1.0),
    ("composite-wave-N400", 0, lambda: W.composite_wave(400), 0, 50.0, 0.4, 6.3, -1.0, 1.0),
    ("burgers-minus-sin-N200", 1, lambda: W.burgers_sine(200, 0.0, -1.0), 0, 50.0, 0.5, 1.5, -1.0, 1.0),
    ("burgers-half-plus-sin-N200", 1, lambda: W.burgers_sine(200, 0.5, 1.0), 0, 50.0, 0.5, 0.55, -1.0, 1.0),
    ("sod-N300", 2, lambda: W.sod(300), 1, 50.0, 0.5, 1.7, -5.0, 5.0),
    ("lax-N300", 2, lambda: W.lax(300), 1, 10.0, 0.5, 1.3, -5.0, 5.0),
    ("123-N300", 2, lambda: W.riemann_123(300), 1, 50.0, 0.5, 1.0, -5.0, 5.0),
    ("shu-osher-N400", 2, lambda: W.shu_osher(400), 1, 50.0, 0.5, 1.8, -5.0, 5.0),
]


@pytest.mark.parametrize("case", VALIDATION, ids=[c[0] for c in VALIDATION])
def test_validation_set_matches_the_oracle(wtlib, oracle, case):
    """The paper's 1D validation problems on its grids to its final times: strict mode bitwise
    equal to the oracle (same step count, same t), fast mode within the L1 tolerance."""
    b, O = wtlib, oracle
    name, flux, make, bc, aR, cfl, tf, lo, hi = case
    U, x, dx = make()
    n = U.shape[1]
    op = O.problem(flux, bc=bc, alpha_R=aR)
    ref, t_ref, s_ref = O.run(op, U, dx, cfl=cfl, t_final=tf)
    grid = b.grid_1d(n, lo, hi)
    u, t, s = _run(b, b.problem(flux, bc=bc, mode=b.WT_MODE_STRICT, alpha_R=aR), U, grid, cfl=cfl, t_final=tf)
    assert t == t_ref == tf and s == s_ref
    assert np.array_equal(u, ref), np.abs(u - ref).max()
    u, t, s = _run(b, b.problem(flux, bc=bc, mode=b.WT_MODE_FAST, alpha_R=aR), U, grid, cfl=cfl, t_final=tf)
    assert abs(t - tf) <= 1e-14 * tf
    l1 = dx * np.abs(u - ref).sum(axis=1)
    assert np.all(l1 <= SHOCK_L1_TOL * np.maximum(1.0, dx * np.abs(ref).sum(axis=1))), l1

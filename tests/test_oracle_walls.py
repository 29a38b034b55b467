"""Pins of the oracle's reflective walls, of its sampled RHS and of its 2D wall fill (no GPU).

A reflective wall (the blast waves of Sec. 4.2, the Rayleigh-Taylor and implosion tests of
Sec. 4.3) sets each ghost cell to the mirror image of the interior with the normal momentum
negated.  What fixes it without restating it:
  - a uniform flow into a wall (and away from the other) is, until the two walls' waves meet,
    the exact Riemann solution of the mirrored states (rho, u, p | rho, -u, p) centred on the
    wall: a reflected shock at one wall, a rarefaction at the other;
  - on data mirrored about the middle of the domain the scheme keeps the mirror symmetry, so
    the wall fluxes of mass and energy vanish and both are conserved to rounding;
  - in 2D, data uniform along the wall equal the 1D run across it.
A planted wrong sign on the normal momentum (an oracle built with one line changed) must
fail the first two.
"""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

T_WALL = 0.2  # before the left rarefaction's head meets the right wall's shock (about t = 0.35)


def _wall_exact(O, x, t, rho=1.0, u=1.0, p=1.0):
    """Uniform flow (rho, u, p), u > 0, in [0, 1] between two walls: the rarefaction of
    (rho, -u, p | rho, u, p) at x = 0 and the shock of (rho, u, p | rho, -u, p) at x = 1."""
    rl, ul, pl = O.riemann_sample((rho, -u, p), (rho, u, p), x, 0.0, t)
    rr, ur, pr = O.riemann_sample((rho, u, p), (rho, -u, p), x, 1.0, t)
    left = x < 0.5
    return np.where(left, rl, rr), np.where(left, ul, ur), np.where(left, pl, pr)


def _wall_run(O, n, alpha_R=10.0):
    x, dx = W.grid_1d(n, 0.0, 1.0, periodic=False)
    U = W.cons_1d(np.ones(n), np.ones(n), np.ones(n))
    P = O.problem(O.FLUX_EULER1D, bc=O.BC_REFLECTIVE, alpha_R=alpha_R)
    u, t, _ = O.run(P, U, dx, cfl=0.5, t_final=T_WALL)
    assert t == T_WALL
    return x, dx, u


def _wall_errors(O, n):
    x, dx, u = _wall_run(O, n)
    rho, vel, p = W.prim_1d(u)
    re, ue, pe = _wall_exact(O, x, T_WALL)
    l1 = dx * np.abs(rho - re).sum()
    tv_all = np.abs(np.diff(rho)).sum() / np.abs(np.diff(re)).sum()
    inner = slice(3, n - 3)  # without the wall-heating layer of three cells at each wall
    tv_inner = np.abs(np.diff(rho[inner])).sum() / np.abs(np.diff(re[inner])).sum()
    return l1, tv_all, tv_inner, dx * np.abs(vel - ue).sum()


def test_the_exact_wall_solution_holds_until_the_waves_meet(oracle):
    """The two mirrored Riemann solutions leave the middle of the domain untouched at T_WALL,
    so gluing them there is the exact solution of the wall problem."""
    xm = np.linspace(0.45, 0.8, 36)  # rarefaction head near 0.437, reflected shock near 0.815
    for k in range(3):
        assert np.allclose(_wall_exact(oracle, xm, T_WALL)[k], 1.0, rtol=0, atol=0)
    # a reflected shock: density and pressure rise at the wall, the gas comes to rest there
    r, u, p = _wall_exact(oracle, np.array([0.999]), T_WALL)
    assert r[0] > 2.0 and p[0] > 2.0 and abs(u[0]) < 1e-12
    r, u, p = _wall_exact(oracle, np.array([0.001]), T_WALL)
    assert r[0] < 0.5 and abs(u[0]) < 1e-12


def test_reflective_walls_against_exact_riemann_solutions(oracle):
    """L1(rho) and L1(u) fall (first order at the shock: at least 1.6x per doubling), no new
    extrema beyond 5% of the exact total variation away from the walls (10% with the wall
    cells, where every shock-capturing scheme shows the wall-heating dip behind a reflected
    shock)."""
    O = oracle
    errs = [_wall_errors(O, n) for n in (200, 400, 800)]
    for (a, *_), (b, *_) in zip(errs, errs[1:]):
        assert b < a / 1.6
    for (a, _, _, ua), (b, _, _, ub) in zip(errs, errs[1:]):
        assert ub < ua / 1.6
    assert errs[-1][0] < 2e-3
    for l1, tv_all, tv_inner, _ in errs:
        assert tv_inner < 1.05 and tv_all < 1.10


def test_planted_wall_sign_fails_the_exact_solution(oracle):
    """The same oracle with the normal momentum's sign kept in the reflective ghosts: the wall
    lets the flow through, and the pin above fails by two orders of magnitude."""
    O = oracle
    with O.using(O.planted("REFLECT_SIGN")):
        l1, tv_all, tv_inner, _ = _wall_errors(O, 200)
    assert l1 > 0.1


def _mirrored_state(n):
    """rho, p, E even and rho u odd about x = 1/2, exactly (the right half is the left half
    reversed)."""
    x, dx = W.grid_1d(n, 0.0, 1.0, periodic=False)
    h = n // 2
    rng = np.random.default_rng(5)
    xl = x[:h]
    r = rng.uniform(size=h)
    rho = 1.0 + 0.3 * np.cos(2 * np.pi * xl) + 0.1 * r
    u = 0.5 * np.sin(2 * np.pi * xl) * (1.0 + 0.2 * r)
    p = 1.0 + 0.2 * r
    Ul = W.cons_1d(rho, u, p)
    U = np.concatenate([Ul, Ul[:, ::-1] * np.array([[1.0], [-1.0], [1.0]])], axis=1)
    return U, dx


def test_reflective_walls_conserve_mass_and_energy_on_mirrored_data(oracle):
    """With data mirrored about the middle, alpha_1 = alpha_3 and each wall interface sees
    mirrored stencils, so its mass and energy fluxes vanish: sum rho and sum E stay constant to
    rounding over 100 steps, and the solution stays mirrored.  A wall that lets mass through
    (the planted sign) changes both by percents."""
    O = oracle
    U, dx = _mirrored_state(200)
    P = O.problem(O.FLUX_EULER1D, bc=O.BC_REFLECTIVE, alpha_R=10.0)
    v, _, steps = O.run(P, U, dx, cfl=0.5, n_steps=100)
    assert steps == 100
    for c in (0, 2):
        assert abs(v[c].sum() - U[c].sum()) <= 1e-13 * U[c].sum()
    assert np.abs(v[0] - v[0][::-1]).max() <= 1e-13 and np.abs(v[1] + v[1][::-1]).max() <= 1e-13
    with O.using(O.planted("REFLECT_SIGN")):
        w, _, _ = O.run(P, U, dx, cfl=0.5, n_steps=100)
    assert abs(w[0].sum() - U[0].sum()) > 1e-3 * U[0].sum()


@pytest.mark.parametrize("wall_dir", [0, 1], ids=["x-walls", "y-walls"])
def test_2d_reflective_walls_equal_the_1d_run(oracle, wall_dir):
    """2D Euler data uniform along the walls, at rest along them, reflective walls across and
    periodic along: every line across the walls equals the 1D run (the same dt), because the
    sweep along the walls sees uniform data and the shear field carries zero."""
    O = oracle
    n, k = 24, 5  # cells across the walls, lines along them
    x, dx = W.grid_1d(n, 0.0, 1.0, periodic=False)
    rng = np.random.default_rng(2)
    rho = 1.0 + 0.4 * rng.uniform(size=x.size)
    vel = rng.uniform(-0.5, 0.5, size=x.size)
    p = 0.5 + rng.uniform(size=x.size)
    U1 = W.cons_1d(rho, vel, p)
    m = U1.shape[1]
    P1 = O.problem(O.FLUX_EULER1D, bc=O.BC_REFLECTIVE, alpha_R=10.0)
    dt = 0.2 * dx
    ref, _, _ = O.run(P1, U1, dx, dt_fixed=dt, n_steps=20)
    zero = np.zeros(m)
    if wall_dir == 1:  # walls at y = 0, 1: the profile runs along y, uniform along x
        U2 = np.stack([np.repeat(U1[0][:, None], k, 1), np.repeat(zero[:, None], k, 1),
                       np.repeat(U1[1][:, None], k, 1), np.repeat(U1[2][:, None], k, 1)])
        P2 = O.problem(O.FLUX_EULER2D, bc=O.BC_PERIODIC, bc_y=O.BC_REFLECTIVE, alpha_R=10.0)
        out, _, _ = O.run(P2, U2, 1.0 / k, dy=dx, dt_fixed=dt, n_steps=20)
        lines = [out[[0, 2, 3], :, i] for i in range(k)]
    else:  # walls at x = 0, 1: the profile runs along x, uniform along y
        U2 = np.stack([np.repeat(U1[0][None, :], k, 0), np.repeat(U1[1][None, :], k, 0),
                       np.repeat(zero[None, :], k, 0), np.repeat(U1[2][None, :], k, 0)])
        P2 = O.problem(O.FLUX_EULER2D, bc=O.BC_REFLECTIVE, bc_y=O.BC_PERIODIC, alpha_R=10.0)
        out, _, _ = O.run(P2, U2, dx, dy=1.0 / k, dt_fixed=dt, n_steps=20)
        lines = [out[[0, 1, 3], j, :] for j in range(k)]
    # the 2D pressure rounds rho (u^2 + v^2) / 2 in another order than the 1D rho u u / 2, so
    # the lines agree to rounding, not bit for bit
    scale = np.abs(ref).max(axis=1, keepdims=True)
    for line in lines:
        assert np.all(np.abs(line - ref) <= 1e-14 * scale), np.abs(line - ref).max()
    tangential = 2 if wall_dir == 0 else 1
    assert np.abs(out[tangential]).max() == 0.0  # still at rest along the walls
    # a 2D wall fill with the planted sign departs from the (pinned) 1D run at once
    with O.using(O.planted("REFLECT_SIGN")):
        bad, _, _ = O.run(P2, U2, *((dx, 1.0 / k) if wall_dir == 0 else (1.0 / k, dx)), dt_fixed=dt, n_steps=20)
    line = bad[[0, 1, 3], 0, :] if wall_dir == 0 else bad[[0, 2, 3], :, 0]
    assert np.abs(line - ref).max() > 1e-2 * np.abs(ref).max()


@pytest.mark.parametrize("case", ["euler1d", "euler2d", "euler2d_gravity", "euler2d_walls"])
def test_rhs_at_equals_rhs(oracle, case):
    """The sampled RHS (used to check the GPU on grids too large for a whole oracle RHS) is the
    whole RHS at every cell, bit for bit, with and without the gravity source."""
    O = oracle
    rng = np.random.default_rng(9)
    if case == "euler1d":
        n = 37
        x, dx = W.grid_1d(n, 0.0, 1.0, periodic=False)
        U = W.cons_1d(0.5 + rng.uniform(size=n), rng.uniform(-1, 1, n), 0.5 + rng.uniform(size=n))
        P = O.problem(O.FLUX_EULER1D, bc=(O.BC_OUTFLOW, O.BC_REFLECTIVE), alpha_R=10.0)
        dy = 1.0
        cells = np.arange(n)
    else:
        nx, ny = 13, 11
        dx, dy = 1.0 / nx, 1.5 / ny
        sh = (ny, nx)
        U = W.cons_2d(0.5 + rng.uniform(size=sh), rng.uniform(-1, 1, sh), rng.uniform(-1, 1, sh),
                      0.5 + rng.uniform(size=sh))
        g = 0.1 if case == "euler2d_gravity" else 0.0
        if case == "euler2d_walls":
            P = O.problem(O.FLUX_EULER2D, bc=O.BC_REFLECTIVE, bc_y=(O.BC_OUTFLOW, O.BC_REFLECTIVE), alpha_R=10.0)
        else:
            P = O.problem(O.FLUX_EULER2D, bc=O.BC_PERIODIC, bc_y=O.BC_REFLECTIVE, alpha_R=50.0, gravity=g)
        cells = np.arange(nx * ny)
    L = O.rhs(P, U, dx, dy)
    at = O.rhs_at(P, U, cells, dx, dy)
    m = U.shape[0]
    assert np.array_equal(at, L.reshape(m, -1).T)
    if case == "euler2d_gravity":  # the source is there: without it the momentum row differs
        P0 = O.problem(O.FLUX_EULER2D, bc=O.BC_PERIODIC, bc_y=O.BC_REFLECTIVE, alpha_R=50.0)
        assert not np.array_equal(O.rhs_at(P0, U, cells, dx, dy)[:, 2], at[:, 2])

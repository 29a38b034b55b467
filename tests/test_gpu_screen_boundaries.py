"""Stencils on either side of the two decisions of a reconstruction: the restriction test of
Eq. (be_res) and the theta switch of Eq. (tau_we6).

The fast policy settles most of these decisions in FP32 under an error bound and computes the
rest in FP64 from stencil differences; the strict policy evaluates them literally.  Here every
designed stencil lies at a relative distance 1e-10 .. 1e-1 from a point where the oracle's
decision changes, in pairs with one stencil on each side, for alpha_R = 50 and 10 and at three
input scales: about 1e-5, where eps = 1e-10 competes with the indicators, about 1, and about
1e3.  One family has beta_3 cancelling to near zero, where the screen's absolute error bound
is the one that matters.

Linear advection with a = +1 or -1 (so alpha = 1) makes the split flux of one side equal to u
and the other zero, so each designed stencil is the whole stencil of one interface: placed
as it is for a = 1, reversed and negated for a = -1 (the mirrored minus side of the flux
splitting, Sec. 2.3).  The RHS must match the oracle (strict bit for bit, fast within 1e-13
normwise), and so must one RK3 step through each launch strategy.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

ALPHAS_R = (50.0, 10.0)
SCALES = {"eps-scale": 1e-5, "unit": 1.0, "large": 1e3}
PAIRS = 100  # boundary points per family and array: 600 stencils, 3600 cells


def _flag(O, q, alpha_r, which):
    v, theta, restricted = O.weno_theta(q, 1e-10, alpha_r)
    return restricted if which in (0, 2) else theta


def _boundary_pairs(O, rng, n, alpha_r, which, scale):
    """n pairs of stencils straddling a change of the oracle's restriction decision
    (which = 0; which = 2 with beta_3 cancelling) or of its theta (which = 1)."""
    out = []
    while len(out) < 2 * n:
        if which == 2:
            a = rng.uniform(0.5, 2.0) * rng.choice([-1.0, 1.0])
            d = np.concatenate([rng.normal(size=2), [a, 1.5 * a, 3.0 * a]])
            u = np.concatenate([[0.0], np.cumsum(d)]) * scale
        else:
            u = rng.normal(size=6) * scale
        v = rng.normal(size=6) * scale * 10 ** rng.uniform(-1, 1)
        f0 = _flag(O, u, alpha_r, which)
        if _flag(O, u + v, alpha_r, which) == f0:
            continue
        lo, hi = 0.0, 1.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if _flag(O, u + mid * v, alpha_r, which) == f0:
                lo = mid
            else:
                hi = mid
        lam = 0.5 * (lo + hi)
        off = 10 ** rng.uniform(-10, -1) * max(lam, 1e-3)
        out.append(u + (lam - off) * v)
        out.append(u + (lam + off) * v)
    return np.array(out)


_CACHE = {}


def _stencils(O, alpha_r, scale_name):
    key = (alpha_r, scale_name)
    if key not in _CACHE:
        rng = np.random.default_rng([int(alpha_r), list(SCALES).index(scale_name), 1504])
        _CACHE[key] = np.concatenate(
            [_boundary_pairs(O, rng, PAIRS, alpha_r, which, SCALES[scale_name]) for which in (0, 1, 2)])
    return _CACHE[key]


def _state(Q, a):
    """One periodic row whose interface 6s + 5/2 has the designed stencil s on its upwind side."""
    seg = Q if a > 0 else -Q[:, ::-1]
    return np.ascontiguousarray(seg.reshape(1, -1))


CASES = [(ar, sc, a) for ar in ALPHAS_R for sc in SCALES for a in (1.0, -1.0)]
IDS = [f"alphaR{int(ar)}-{sc}-a{'+' if a > 0 else '-'}" for ar, sc, a in CASES]


def test_boundary_stencils_straddle_the_oracle_decisions(oracle):
    """The generator's own claim, on the CPU: each pair falls on both sides of the decision it
    was built for, and most pairs lie close to it."""
    O = oracle
    for alpha_r in ALPHAS_R:
        Q = _stencils(O, alpha_r, "unit")
        for f, which in enumerate((0, 1, 2)):
            P = Q[2 * PAIRS * f:2 * PAIRS * (f + 1)]
            flags = np.array([_flag(O, q, alpha_r, which) for q in P])
            assert np.all(flags[0::2] != flags[1::2])
            assert np.median(np.abs(P[0::2] - P[1::2]).max(axis=1) / np.abs(P).max()) < 1e-3


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_rhs_at_decision_boundaries(wtlib, oracle, case):
    b, O = wtlib, oracle
    alpha_r, scale_name, a = case
    U = _state(_stencils(O, alpha_r, scale_name), a)
    n = U.shape[1]
    dx = 2.0 / n
    ref = O.rhs(O.problem(O.FLUX_ADVECTION, adv_speed=a, alpha_R=alpha_r, bc=O.BC_PERIODIC), U, dx)
    g = b.grid_1d(n, -1.0, 1.0)
    for mode in (b.WT_MODE_STRICT, b.WT_MODE_FAST):
        prob = b.problem(b.WT_FLUX_ADVECTION, adv_speed=a, alpha_R=alpha_r, bc=b.WT_BC_PERIODIC, mode=mode)
        ws = b.alloc_workspace(b.workspace_bytes(prob, g))
        u = torch.from_numpy(U).cuda()
        L = torch.full_like(u, np.nan)
        b.weno_theta_rhs(prob, g, u, L, ws)
        torch.cuda.synchronize()
        Lg = L.cpu().numpy()
        if mode == b.WT_MODE_STRICT:
            assert np.array_equal(Lg, ref), np.abs(Lg - ref).max()
        else:
            err = np.abs(Lg - ref).max()
            assert err <= 1e-13 * np.abs(ref).max(), err / np.abs(ref).max()


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_one_step_at_decision_boundaries(wtlib, oracle, case):
    """One RK3 step at CFL 0.5: the step-blocked kernel (chosen automatically for 3600 cells)
    and the per-stage kernels."""
    b, O = wtlib, oracle
    alpha_r, scale_name, a = case
    U = _state(_stencils(O, alpha_r, scale_name), a)
    n = U.shape[1]
    dx = 2.0 / n
    ref, _, _ = O.run(O.problem(O.FLUX_ADVECTION, adv_speed=a, alpha_R=alpha_r, bc=O.BC_PERIODIC), U, dx, cfl=0.5,
                      n_steps=1)
    g = b.grid_1d(n, -1.0, 1.0)
    for mode in (b.WT_MODE_STRICT, b.WT_MODE_FAST):
        for launch in (b.WT_LAUNCH_AUTO, b.WT_LAUNCH_STAGES):
            prob = b.problem(b.WT_FLUX_ADVECTION, adv_speed=a, alpha_R=alpha_r, bc=b.WT_BC_PERIODIC, mode=mode,
                             launch=launch)
            ws = b.alloc_workspace(b.workspace_bytes(prob, g))
            u = torch.from_numpy(U).cuda()
            t, steps = b.weno_theta_step(prob, g, u, 0.5, ws, max_steps=1)
            assert steps == 1
            ug = u.cpu().numpy()
            if mode == b.WT_MODE_STRICT:
                assert np.array_equal(ug, ref), (launch, np.abs(ug - ref).max())
            else:
                err = np.abs(ug - ref).max()
                assert err <= 1e-13 * np.abs(ref).max(), (launch, err / np.abs(ref).max())

"""The oracle's WENO-theta reconstruction against the same formulas evaluated in exact rational
arithmetic, on the CPU.

Each double input is converted exactly to a fraction; the sub-stencil values of
Eqs. (fh0)-(fh3), the indicators of Eqs. (be0_cen)-(be3_cen), the restriction of Eq. (be_res),
tau5 and tau6 of Eqs. (tau_5), (tau_6), the switch of Eq. (tau_we6), the linear weights of
Eq. (gam_we6) and the nonlinear weights of Eqs. (om), (fh_nonlinear) are then evaluated without
rounding.  The oracle, in binary64, must take the same two decisions wherever the exact
margin of a decision exceeds what rounding the indicators can move (a bound from 1e-13 of
the largest input), and its value must lie within rounding of the exact one.  The same
comparison runs over the whole right-hand side of Eq. (mod_semi) for periodic linear
advection on grids of 3 to 8 cells (a = +1 and -1, so both the plus side and the mirrored
minus side of the flux splitting carry the data).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

EPS = 1e-10


def exact_weno(q, eps=EPS, alpha_r=50.0):
    """(value, theta, restricted, near a restriction tie, near a theta tie, max |fh_k|) of one
    reconstruction from six split-flux values q_0..q_5 = f_{j-2}..f_{j+3}, in exact
    arithmetic."""
    f = [Fr(float(v)) for v in q]
    e, ar = Fr(eps), Fr(alpha_r)
    fh = [
        Fr(2, 6) * f[0] - Fr(7, 6) * f[1] + Fr(11, 6) * f[2],   # Eq. (fh0)
        -Fr(1, 6) * f[1] + Fr(5, 6) * f[2] + Fr(2, 6) * f[3],   # Eq. (fh1)
        Fr(2, 6) * f[2] + Fr(5, 6) * f[3] - Fr(1, 6) * f[4],    # Eq. (fh2)
        Fr(11, 6) * f[3] - Fr(7, 6) * f[4] + Fr(2, 6) * f[5],   # Eq. (fh3)
    ]
    beta = [
        Fr(13, 12) * (f[0] - 2 * f[1] + f[2]) ** 2 + (f[0] - 3 * f[1] + 2 * f[2]) ** 2,        # (be0_cen)
        Fr(13, 12) * (f[1] - 2 * f[2] + f[3]) ** 2 + (f[3] - f[2]) ** 2,                       # (be1_cen)
        Fr(13, 12) * (f[2] - 2 * f[3] + f[4]) ** 2 + (f[2] - f[3]) ** 2,                       # (be2_cen)
        Fr(13, 48) * (3 * f[2] - 7 * f[3] + 5 * f[4] - f[5]) ** 2
        + (2 * f[3] - 3 * f[4] + f[5]) ** 2,                                                   # (be3_cen)
    ]
    tau5 = Fr(13, 12) * (f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4]) ** 2 \
        + (-f[1] + 3 * f[2] - 3 * f[3] + f[4]) ** 2                                            # (tau_5)
    tau6 = Fr(13, 12) * (-f[0] + 5 * f[1] - 10 * f[2] + 10 * f[3] - 5 * f[4] + f[5]) ** 2 \
        + Fr(1, 4) * (f[0] - 3 * f[1] + 2 * f[2] + 2 * f[3] - 3 * f[4] + f[5]) ** 2          # (tau_6)
    theta = 0 if tau6 < tau5 else 1                                                            # (tau_we6)
    tau = tau6 if theta == 0 else tau5
    # R(beta) <= alpha_R with a positive denominator, Eq. (be_res)
    bmax, bmin = max(beta), min(beta)
    restricted = bmax <= ar * (e + bmin)
    if restricted:
        beta = [Fr(0)] * 4
    gam = [Fr(1, 20) * (1 + theta), Fr(3, 20) * (3 + theta), Fr(3, 20) * (3 - theta), Fr(1, 20) * (1 - theta)]
    alpha = [g * (1 + tau / (e + b)) for g, b in zip(gam, beta)]                               # (om)
    s = sum(alpha)
    value = sum(a / s * h for a, h in zip(alpha, fh))                                          # (fh_nonlinear)
    # Either decision may go the other way in binary64 when its exact margin is within the
    # rounding of the indicators: each difference combination is off by a few ulps of the
    # largest input S, so an indicator b = x^2 + y^2 by about 2 E sqrt(b) + E^2, E ~ 1e-13 S
    E = Fr(1, 10 ** 13) * max(abs(v) for v in f)
    sq = lambda v: Fr(float(v) ** 0.5)  # noqa: E731  (a bound, not an exact root)
    near_r = abs(bmax - ar * (e + bmin)) <= 4 * E * (sq(bmax) + ar * sq(bmin)) + 4 * (1 + ar) * E * E
    near_t = abs(tau6 - tau5) <= 4 * E * (sq(tau5) + sq(tau6)) + 4 * E * E
    return value, theta, restricted, near_r, near_t, max(abs(h) for h in fh)


def _stencils(rng, n):
    x = np.arange(6.0)
    out = [rng.normal(size=6) * 10 ** rng.uniform(-6, 3) for _ in range(n)]                 # random
    for _ in range(n):                                                                         # smooth
        h, w, ph, a = 10 ** rng.uniform(-3, -0.5), rng.uniform(0.5, 3), rng.uniform(0, 6.3), 10 ** rng.uniform(-4, 1)
        out.append(a * np.sin(w * h * x + ph) + rng.uniform(-1, 1))
    for _ in range(n):                                                                         # a jump
        k = rng.integers(1, 6)
        out.append(np.where(x < k, rng.uniform(-1, 1), rng.uniform(-1, 1)) + 1e-3 * rng.normal(size=6))
    for _ in range(n // 4):                                                                    # constant, polynomial
        c = rng.uniform(-1, 1, 3)
        out.append(np.full(6, c[0]))
        out.append(c[0] + c[1] * x + c[2] * x * x)
    return out


@pytest.mark.parametrize("alpha_r", [50.0, 10.0])
def test_reconstruction_matches_exact_arithmetic(oracle, alpha_r):
    O = oracle
    rng = np.random.default_rng(int(alpha_r))
    compared = 0
    seen = set()
    for q in _stencils(rng, 150):
        q = np.asarray(q, dtype=np.float64)
        v, theta, restricted = O.weno_theta(q, EPS, alpha_r)
        ex, th_ex, rs_ex, near_r, near_t, scale = exact_weno(q, EPS, alpha_r)
        if near_r or near_t:
            continue  # a near-tie: binary64 may decide either way
        assert (theta, bool(restricted)) == (th_ex, rs_ex), (q, theta, restricted, th_ex, rs_ex)
        err = abs(Fr(v) - ex)
        assert err <= Fr(1, 10 ** 13) * (scale + abs(ex)) + Fr(1, 10 ** 300), (q, float(err))
        compared += 1
        seen.add((th_ex, rs_ex))
    assert compared >= 400
    assert len(seen) == 4  # every combination of the two decisions occurred


@pytest.mark.parametrize("a", [1.0, -1.0])
def test_tiny_periodic_rhs_matches_exact_arithmetic(oracle, a):
    """L_j = -(F_{j+1/2} - F_{j-1/2}) / dx (Eq. (mod_semi)) with the global Lax-Friedrichs
    split of f = a u, alpha = |a| (Eq. (flux_split_lf)): one side is u, the other zero, the
    minus side read mirrored."""
    O = oracle
    rng = np.random.default_rng(7 if a > 0 else 8)
    checked = 0
    for n in range(3, 9):
        for _ in range(6):
            u = rng.normal(size=n) * 10 ** rng.uniform(-3, 1)
            dx = 2.0 / n
            L = O.rhs(O.problem(O.FLUX_ADVECTION, adv_speed=a, bc=O.BC_PERIODIC), u[None, :], dx)[0]
            F = []
            near_tie = False
            for j in range(n):  # interface j + 1/2
                if a > 0:
                    stencil = [u[(j - 2 + k) % n] for k in range(6)]  # v+ = u
                else:
                    stencil = [-u[(j + 3 - k) % n] for k in range(6)]  # v- = -u, mirrored
                val, _, _, near_r, near_t, _ = exact_weno(stencil)
                near_tie |= near_r or near_t
                F.append(val)
            if near_tie:
                continue
            Lex = [-(F[j] - F[j - 1]) / Fr(dx) for j in range(n)]
            scale = max(abs(v) for v in Lex) + max(abs(Fr(float(x))) for x in u) / Fr(dx)
            for j in range(n):
                assert abs(Fr(L[j]) - Lex[j]) <= Fr(1, 10 ** 13) * scale, (n, j, L[j], float(Lex[j]))
            checked += 1
    assert checked >= 30


def test_exact_ties_take_theta_one(oracle):
    """tau6 = tau5 exactly (constant data, and integer data on a line, whose third and higher
    differences vanish in binary64 too): Eq. (tau_we6) takes theta = 1 on the tie, and the
    stencil is restricted (R = 0 or R = 1/(eps + 1), both below alpha_R)."""
    O = oracle
    x = np.arange(6.0)
    for q in (np.full(6, 0.0), np.full(6, 3.25), np.full(6, -7.0), x, 4.0 * x - 9.0, -2.0 * x + 1.0):
        v, theta, restricted = O.weno_theta(q, EPS, 50.0)
        ex, th_ex, rs_ex, _, _, _ = exact_weno(q, EPS, 50.0)
        assert (theta, bool(restricted)) == (1, True) == (th_ex, rs_ex)
        assert Fr(v) == ex  # the interface value of the line, exactly

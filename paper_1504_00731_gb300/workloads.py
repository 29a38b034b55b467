"""Seeded synthetic inputs for the WENO-theta workloads.

This module only builds initial data (grids, seeded random parameters and the
conversion from primitive (rho, u, p) to conserved variables).  It holds none of
the scheme's arithmetic, so the oracle and the CUDA path can both consume it.

Grids (a reading of Sec. 2, where x_j = x_l + j dx is not tied to a point count):
N unknowns, dx = (x_r - x_l) / N.  Periodic problems use the nodes
x_j = x_l + j dx (j = 0..N-1, x_N identified with x_0), which reproduces Table 1;
non-periodic problems use cell centres x_j = x_l + (j + 1/2) dx.

Arrays are float64, component-major: (m, n) in 1D, (m, ny, nx) in 2D (x fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
# alpha_R of Eq. (be_res) for the seeded Riemann workloads.  Reading: the paper takes
# alpha_R small when shocks are present (10 for its Lax and blast-wave tests, 50 for Sod);
# the seeded data here hold density and pressure jumps of up to 10x, and with 50 some of
# them (e.g. problem 1994 of the seed-0 batch) break down at the contact in both the oracle
# and the GPU path, while 10 keeps all of them finite.
ALPHA_R_SEEDED = 10.0


def grid_1d(n: int, lo: float, hi: float, periodic: bool):
    dx = (hi - lo) / n
    j = np.arange(n, dtype=np.float64)
    x = lo + j * dx if periodic else lo + (j + 0.5) * dx
    return x, dx


def cons_1d(rho, u, p, gamma=GAMMA):
    """(rho, u, p) -> (rho, rho u, E), E = p/(gamma-1) + rho u^2 / 2 (Sec. 4.2)."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def cons_2d(rho, u, v, p, gamma=GAMMA):
    """(rho, u, v, p) -> (rho, rho u, rho v, E) (Sec. 4.3)."""
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def prim_1d(U, gamma=GAMMA):
    rho = U[0]
    u = U[1] / rho
    p = (gamma - 1.0) * (U[2] - 0.5 * rho * u * u)
    return rho, u, p


# --------------------------------------------------------------------------------------------
# Scalar advection u_t + u_x = 0 on [-1, 1], periodic
# --------------------------------------------------------------------------------------------

def advection_sine(n: int):
    """u0 = sin(pi x) on [-1, 1] (Eq. (sca_ini_1)); returns (u (1, n), x, dx)."""
    x, dx = grid_1d(n, -1.0, 1.0, periodic=True)
    return np.sin(np.pi * x)[None, :], x, dx


def advection_seeded(n: int, seed: int):
    """u0 = sum_{k=1..3} a_k sin(k pi x + phi_k), a_k ~ U[0,1], phi_k ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 1.0, 3)
    phi = rng.uniform(0.0, 2.0 * np.pi, 3)
    x, dx = grid_1d(n, -1.0, 1.0, periodic=True)
    u = sum(a[k] * np.sin((k + 1) * np.pi * x + phi[k]) for k in range(3))
    return u[None, :], x, dx, (a, phi)


def advection_ic2(n: int, k: int):
    """u0 = (x + 1/2)^k exp(-100 (x + 1/2)^2) (Eq. (sca_ini_2))."""
    x, dx = grid_1d(n, -1.0, 1.0, periodic=True)
    return ((x + 0.5) ** k * np.exp(-100.0 * (x + 0.5) ** 2))[None, :], x, dx


# --------------------------------------------------------------------------------------------
# 1D Euler: seeded Riemann data plus an entropy wave on the right state
# --------------------------------------------------------------------------------------------

@dataclass
class RiemannParams:
    rhoL: float
    uL: float
    pL: float
    rhoR: float
    uR: float
    pR: float
    x0: float
    k: float
    amp: float = 0.2


def riemann_params(seed: int) -> RiemannParams:
    """rho, p ~ U[0.1, 1], u ~ U[-1, 1] on each side, jump x0 ~ U[-1, 1], wave number k ~ U[3, 8]."""
    rng = np.random.default_rng(seed)
    rhoL, rhoR = rng.uniform(0.1, 1.0, 2)
    pL, pR = rng.uniform(0.1, 1.0, 2)
    uL, uR = rng.uniform(-1.0, 1.0, 2)
    x0 = rng.uniform(-1.0, 1.0)
    k = rng.uniform(3.0, 8.0)
    return RiemannParams(rhoL, uL, pL, rhoR, uR, pR, x0, k)


def euler_riemann(n: int, prm: RiemannParams, lo=-5.0, hi=5.0, periodic=False, gamma=GAMMA):
    """Riemann data with the right-side density modulated as rho_R (1 + amp sin(k x)).

    Reading: the additive form rho += 0.2 sin(kx) can make rho negative for rho_R < 0.2,
    so the modulation is multiplicative (the form of the shock/entropy-wave test of Sec. 4.2, TEST 4)."""
    x, dx = grid_1d(n, lo, hi, periodic)
    left = x < prm.x0
    rho = np.where(left, prm.rhoL, prm.rhoR * (1.0 + prm.amp * np.sin(prm.k * x)))
    u = np.where(left, prm.uL, prm.uR)
    p = np.where(left, prm.pL, prm.pR)
    return cons_1d(rho, u, p, gamma), x, dx


def euler_c2(n: int = 4096, seed: int = 0):
    """1D Euler, N = 4096 on [-5, 5], outflow, seeded Riemann + entropy-wave data."""
    return euler_riemann(n, riemann_params(seed))


def sod(n: int, lo=-5.0, hi=5.0):
    """Sod data as printed in Sec. 4.2 (TEST 3) (dense gas on the right): (0.125, 0, 0.1) | (1, 0, 1), jump at 0."""
    x, dx = grid_1d(n, lo, hi, periodic=False)
    left = x < 0.0
    rho = np.where(left, 0.125, 1.0)
    p = np.where(left, 0.1, 1.0)
    return cons_1d(rho, np.zeros(n), p), x, dx


def entropy_wave(n: int, amp=0.2, lo=-1.0, hi=1.0):
    """rho = 1 + amp sin(pi x), u = 1, p = 1, periodic on [-1, 1]: exact solution is translation."""
    x, dx = grid_1d(n, lo, hi, periodic=True)
    return cons_1d(1.0 + amp * np.sin(np.pi * x), np.ones(n), np.ones(n)), x, dx


def symmetric_123(n: int, lo=-5.0, hi=5.0):
    """Mirror-symmetric 123-type data (Sec. 4.2, TEST 3): rho, p even and u odd about the
    domain centre, bit for bit (the right half is the mirror image of the left half; n even)."""
    assert n % 2 == 0
    x, dx = grid_1d(n, lo, hi, periodic=False)
    xl = x[: n // 2]
    rho = 1.0 + 0.1 * np.cos(3.0 * xl)
    u = -2.0 * (1.0 - np.exp(-xl * xl))
    p = 0.4 + 0.05 * np.cos(2.0 * xl)
    rho = np.concatenate([rho, rho[::-1]])
    u = np.concatenate([u, -u[::-1]])
    p = np.concatenate([p, p[::-1]])
    return cons_1d(rho, u, p), x, dx


# --------------------------------------------------------------------------------------------
# Batched 1D Euler: many independent problems of uneven length
# --------------------------------------------------------------------------------------------

@dataclass
class Batch:
    lengths: np.ndarray      # int64 [nprob]
    offsets: np.ndarray      # int64 [nprob], start of each problem in the packed arrays
    bc: np.ndarray           # int32 [nprob], 0 periodic, 1 outflow (both ends)
    dx: np.ndarray           # float64 [nprob]
    lo: np.ndarray
    hi: np.ndarray
    u: np.ndarray            # float64 [3, sum(lengths)] packed, problem p at offsets[p]
    params: list = field(default_factory=list)


def batch_lengths(nprob: int, seed: int, nmin=256, nmax=65536):
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), nprob))).astype(np.int64)


def euler_batch(nprob: int, seed: int, nmin=256, nmax=65536, lengths=None, amp_scale=None, problems=None):
    """Seeded batch: lengths log-uniform in [nmin, nmax], boundary periodic or outflow by coin flip,
    Riemann + entropy-wave data with per-problem seeds (seed * 1_000_003 + p).

    ``problems`` (indices into the nprob problems of the seed, default all) builds only those
    problems, packed in the given order: one rank's share of a partitioned batch.  The draws
    are prefix-stable, so the first k problems of a larger batch are those of a k-problem one."""
    if lengths is None:
        lengths = batch_lengths(nprob, seed, nmin, nmax)
    lengths = np.asarray(lengths, dtype=np.int64)
    rng = np.random.default_rng(seed + 7)
    bc = rng.integers(0, 2, nprob).astype(np.int32)
    ids = np.arange(nprob) if problems is None else np.asarray(problems, dtype=np.int64)
    lengths, bc = lengths[ids], bc[ids]
    k = len(ids)
    offsets = np.zeros(k, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)[:-1]
    u = np.empty((3, int(lengths.sum())))
    dx = np.empty(k)
    params = []
    for i, p in enumerate(ids):
        prm = riemann_params(seed * 1_000_003 + int(p))
        if amp_scale is not None:
            s = amp_scale[p]
            prm = RiemannParams(prm.rhoL * s[0], prm.uL, prm.pL * s[1], prm.rhoR * s[2], prm.uR, prm.pR * s[3],
                                prm.x0, prm.k, prm.amp * s[4])
        U, x, d = euler_riemann(int(lengths[i]), prm, periodic=bool(bc[i] == 0))
        u[:, offsets[i]:offsets[i] + lengths[i]] = U
        dx[i] = d
        params.append(prm)
    return Batch(lengths, offsets, bc, dx, np.full(k, -5.0), np.full(k, 5.0), u, params)


def amplitude_perturbation(nprob: int, seed: int, rel=0.01):
    """Per-problem factors (1 + rel U[-1, 1]) for (rhoL, pL, rhoR, pR, wave amplitude)."""
    rng = np.random.default_rng(seed + 11)
    return 1.0 + rel * rng.uniform(-1.0, 1.0, (nprob, 5))


def adjoint_batch(nprob: int = 256, n: int = 16384, seed: int = 0, perturbed: bool = False):
    """Initial data of the adjoint workload, (nprob, 3, n): nprob 1D Euler problems of n cells on
    [-5, 5] (outflow), Riemann + entropy-wave data with per-problem seeds seed * 1_000_003 + p.
    perturbed=True gives the target's initial data: the jump states' density and pressure and
    the entropy-wave amplitude scaled by (1 + 0.01 U[-1, 1]) per problem."""
    scale = amplitude_perturbation(nprob, seed) if perturbed else None
    U = np.empty((nprob, 3, n))
    dx = 0.0
    for p in range(nprob):
        prm = riemann_params(seed * 1_000_003 + p)
        if scale is not None:
            s = scale[p]
            prm = RiemannParams(prm.rhoL * s[0], prm.uL, prm.pL * s[1], prm.rhoR * s[2], prm.uR, prm.pR * s[3],
                                prm.x0, prm.k, prm.amp * s[4])
        U[p], _, dx = euler_riemann(n, prm)
    return U, dx


# --------------------------------------------------------------------------------------------
# 2D Euler: four Riemann quadrants plus isentropic vortices, periodic on [0, 1]^2
# --------------------------------------------------------------------------------------------

def euler2d_vortices(nx: int, ny: int, seed: int, n_vortex=8, rc=0.05, gamma=GAMMA):
    """Quadrant states rho, p ~ U[0.1, 1], u, v ~ U[-0.5, 0.5] split at (0.5, 0.5), plus n_vortex
    isentropic vortices (strength ~ U[1, 5], centre ~ U[0, 1]^2, core radius rc).

    Reading (synthetic data, no physics claim): with r the distance to a vortex centre over rc,
    du = (b / 2 pi) e^{(1 - r^2)/2} (-(y - yc)/rc), dv = (b / 2 pi) e^{(1 - r^2)/2} ((x - xc)/rc),
    dT = -(gamma - 1) b^2 / (8 gamma pi^2) e^{1 - r^2}; T = T_q max(1 + sum dT, 0.2),
    rho = rho_q (T / T_q)^{1/(gamma - 1)}, p = rho T.  Periodic images are ignored."""
    rng = np.random.default_rng(seed)
    q_rho = rng.uniform(0.1, 1.0, 4)
    q_p = rng.uniform(0.1, 1.0, 4)
    q_u = rng.uniform(-0.5, 0.5, 4)
    q_v = rng.uniform(-0.5, 0.5, 4)
    beta = rng.uniform(1.0, 5.0, n_vortex)
    cen = rng.uniform(0.0, 1.0, (n_vortex, 2))
    dx, dy = 1.0 / nx, 1.0 / ny
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)  # (ny, nx)
    quad = (X >= 0.5).astype(np.int64) + 2 * (Y >= 0.5).astype(np.int64)
    rho_q, p_q = q_rho[quad], q_p[quad]
    T_q = p_q / rho_q
    du = np.zeros_like(X)
    dv = np.zeros_like(X)
    dT = np.zeros_like(X)
    for i in range(n_vortex):
        rx = (X - cen[i, 0]) / rc
        ry = (Y - cen[i, 1]) / rc
        r2 = rx * rx + ry * ry
        e = np.exp(0.5 * (1.0 - r2))
        du += beta[i] / (2 * np.pi) * e * (-ry)
        dv += beta[i] / (2 * np.pi) * e * rx
        dT += -(gamma - 1.0) * beta[i] ** 2 / (8 * gamma * np.pi ** 2) * e * e
    T = T_q * np.maximum(1.0 + dT, 0.2)
    rho = rho_q * (T / T_q) ** (1.0 / (gamma - 1.0))
    p = rho * T
    u = q_u[quad] + du
    v = q_v[quad] + dv
    return cons_2d(rho, u, v, p, gamma), dx, dy


# --------------------------------------------------------------------------------------------
# Test problems of Sec. 4.2 / 4.3 that run on the existing kernels (reflective walls, gravity)
# --------------------------------------------------------------------------------------------
def blast_waves(n: int):
    """Two interacting blast waves, Eq. (blast_prob) (TEST 5): (rho, u, p) = (1, 0, 1000) on
    (0, 0.1), (1, 0, 0.01) on (0.1, 0.9), (1, 0, 100) on (0.9, 1); reflective walls at both
    ends; the paper takes alpha_R = 10 and t = 0.038 on N = 801."""
    x, dx = grid_1d(n, 0.0, 1.0, periodic=False)
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    return cons_1d(np.ones(n), np.zeros(n), p), x, dx


RT_GRAVITY = 0.1


def rayleigh_taylor(nx: int, ny: int, g=RT_GRAVITY, gamma=GAMMA):
    """Rayleigh-Taylor instability (TEST 6, Sec. 4.3) on (-0.25, 0.25) x (-0.75, 0.75): rho = 2
    for y >= 0 and 1 below, hydrostatic p = 2.5 - rho g y, u = 0,
    v = (0.01 / 4)(1 + cos 4 pi x)(1 + cos(4 pi y / 3)); periodic in x, reflective in y, source
    terms with g = 0.1.  Cell centres, so the data are mirror-symmetric about x = 0."""
    x, dx = grid_1d(nx, -0.25, 0.25, periodic=False)
    x = 0.5 * (x - x[::-1])  # exactly antisymmetric cell centres
    y, dy = grid_1d(ny, -0.75, 0.75, periodic=False)
    X, Y = np.meshgrid(x, y)
    rho = np.where(Y >= 0.0, 2.0, 1.0)
    p = 2.5 - rho * g * Y
    v = 0.0025 * (1.0 + np.cos(4.0 * np.pi * X)) * (1.0 + np.cos(4.0 * np.pi * Y / 3.0))
    return cons_2d(rho, np.zeros_like(X), v, p, gamma), dx, dy


def implosion(n: int, gamma=GAMMA):
    """Implosion problem, Eq. (eu2D_im) (TEST 7) on (0, 1)^2: (rho, p) = (1, 1) for
    x + y > 1/2 and (0.125, 0.14) otherwise, at rest, reflective walls; the paper takes
    alpha_R = 1 and t = 5 on 400 x 400.  Symmetric about the diagonal x = y."""
    x, dx = grid_1d(n, 0.0, 1.0, periodic=False)
    X, Y = np.meshgrid(x, x)
    inner = X + Y > 0.5
    rho = np.where(inner, 1.0, 0.125)
    p = np.where(inner, 1.0, 0.14)
    return cons_2d(rho, np.zeros_like(X), np.zeros_like(X), p, gamma), dx, dx


# --------------------------------------------------------------------------------------------
# The remaining 1D validation set of Sec. 3.3 / 4.1 / 4.2
# --------------------------------------------------------------------------------------------
def sine_max(n: int):
    """u0 = max(sin pi x, 0) on (-1, 1), periodic (Eq. (sca_ini_3), resolution test)."""
    x, dx = grid_1d(n, -1.0, 1.0, periodic=True)
    return np.maximum(np.sin(np.pi * x), 0.0)[None, :], x, dx


def composite_wave(n: int):
    """Gaussian, square wave, triangle and semi-ellipse (Eq. (sca_ini_4), TEST 1) on (-1, 1),
    periodic; z = -0.7, delta = 0.005, beta = log 2 / (36 delta^2), a = 0.5, alpha = 10."""
    x, dx = grid_1d(n, -1.0, 1.0, periodic=True)
    return composite_wave_at(x)[None, :], x, dx


def composite_wave_at(x):
    z, d, a, al = -0.7, 0.005, 0.5, 10.0
    beta = np.log(2.0) / (36.0 * d * d)
    G = lambda zz: np.exp(-beta * (x - zz) ** 2)
    F = lambda aa: np.sqrt(np.maximum(1.0 - al * al * (x - aa) ** 2, 0.0))
    u = np.zeros_like(x)
    m = (x >= -0.8) & (x <= -0.6)
    u[m] = ((G(z - d) + 4.0 * G(z) + G(z + d)) / 6.0)[m]
    u[(x >= -0.4) & (x <= -0.2)] = 1.0
    m = (x >= 0.0) & (x <= 0.2)
    u[m] = (1.0 - np.abs(10.0 * (x - 0.1)))[m]
    m = (x >= 0.4) & (x <= 0.6)
    u[m] = ((F(a - d) + 4.0 * F(a) + F(a + d)) / 6.0)[m]
    return u


def burgers_sine(n: int, shift=0.0, sign=-1.0):
    """Burgers data of TEST 2: u0 = -sin(pi x) (Eq. (bur_ini_1)) or 1/2 + sin(pi x)
    (Eq. (bur_ini_2), shift = 0.5, sign = 1) on (-1, 1), periodic."""
    x, dx = grid_1d(n, -1.0, 1.0, periodic=True)
    return (shift + sign * np.sin(np.pi * x))[None, :], x, dx


def lax(n: int, lo=-5.0, hi=5.0):
    """Lax's problem (Eq. (lax_prob), TEST 3): (0.445, 0.698, 3.528) | (0.5, 0, 0.571) at 0."""
    x, dx = grid_1d(n, lo, hi, periodic=False)
    left = x < 0.0
    return cons_1d(np.where(left, 0.445, 0.5), np.where(left, 0.698, 0.0), np.where(left, 3.528, 0.571)), x, dx


def shu_osher(n: int, lo=-5.0, hi=5.0):
    """Shu-Osher shock / density-wave interaction (Eq. (shock_den_prob), TEST 4):
    (3.857143, 2.629369, 31/3) on (-5, -4), (1 + 0.2 sin 5x, 0, 1) beyond, zero gradient."""
    x, dx = grid_1d(n, lo, hi, periodic=False)
    left = x < -4.0
    rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    return cons_1d(rho, np.where(left, 2.629369, 0.0), np.where(left, 31.0 / 3.0, 1.0)), x, dx


def riemann_123(n: int, lo=-5.0, hi=5.0):
    """The 123 problem as printed (Eq. (123_prob), TEST 3): (1, -2, 0.4) | (1, 2, 0.4) at 0."""
    x, dx = grid_1d(n, lo, hi, periodic=False)
    left = x < 0.0
    return cons_1d(np.ones(n), np.where(left, -2.0, 2.0), np.full(n, 0.4)), x, dx


def ulp_perturbed(U, seed: int):
    """The data with every value moved by at most one unit in its last place (seeded): the
    input of a second oracle run that shows how far rounding alone carries two evaluations of
    the method apart (amplified by the flow, or flipping a decision that sits on its threshold)."""
    U = np.asarray(U, dtype=np.float64)
    rng = np.random.default_rng(seed)
    return U * (1.0 + rng.integers(-1, 2, U.shape) * 2.0 ** -52)

"""The discrete adjoint at the adjoint workload's shape and length.

The workload: 256 1D Euler problems of 16384 cells (outflow, seeded Riemann + entropy-wave
data), 1024 RK steps with checkpoints every 32, loss J = (dx / 2) sum_p sum_j (rho_pj(T) -
rho*_pj)^2 against a target run from data whose jump states and wave amplitude are scaled by
(1 + 0.01 U[-1, 1]).  The gradient is the reverse mode of the exact map the forward computes
(Eqs. (3rd_RK), (mod_semi), (fh_nonlinear), with theta, the restriction and the maxima frozen
where the forward took them).
"""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, K, CFL = 16384, 32, 0.5


def _forward(b, prob, U, steps):
    """rho(T) of every problem, through the batched entry point."""
    nprob = U.shape[0]
    segs = []
    for p in range(nprob):
        s = b.WtSegment()
        s.offset, s.n, s.lo, s.hi, s.bc_lo, s.bc_hi = p * N, N, -5.0, 5.0, 1, 1
        segs.append(s)
    ws = b.alloc_workspace(b.workspace_bytes(prob, None, nprob * N, nprob))
    u = torch.from_numpy(np.ascontiguousarray(U.transpose(1, 0, 2).reshape(3, nprob * N))).cuda()
    b.weno_theta_step_batched(prob, segs, u, nprob * N, CFL, steps, ws)
    return u[0].reshape(nprob, N).cpu().numpy()


def _adjoint(b, prob, U0, target, steps, dx):
    nprob = U0.shape[0]
    g = b.grid_1d(N, -5.0, 5.0)
    ws = b.alloc_workspace(b.adjoint_workspace_bytes(prob, g, nprob, steps, K))
    u0 = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
    gT, g0, uT = torch.zeros_like(u0), torch.empty_like(u0), torch.empty_like(u0)
    b.weno_theta_adjoint(prob, g, nprob, u0, CFL, steps, K, gT, g0, ws, uT=uT)  # u(T) first
    gT[:, 0, :] = dx * (uT[:, 0, :] - torch.from_numpy(target).cuda())
    b.weno_theta_adjoint(prob, g, nprob, u0, CFL, steps, K, gT, g0, ws, uT=uT)
    torch.cuda.synchronize()
    return g0.cpu().numpy(), uT.cpu().numpy()


def test_adjoint_full_length_strict_matches_dual_numbers(wtlib, oracle):
    """Problem 0 of the workload, all 1024 steps with checkpoints every 32 (31 of 32 segments
    recomputed), strict mode: u(T) equals the oracle's bit for bit, and <g, d> equals the
    oracle's forward-mode (dual-number) derivative of the same map to 1e-9 relative."""
    b, O = wtlib, oracle
    steps = 1024
    U0, dx = W.adjoint_batch(1, N)
    Ut, _ = W.adjoint_batch(1, N, perturbed=True)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, mode=b.WT_MODE_STRICT, alpha_R=W.ALPHA_R_SEEDED)
    target = _forward(b, prob, Ut, steps)
    g0, uT = _adjoint(b, prob, U0, target, steps, dx)
    d = np.random.default_rng(3).standard_normal((3, N))
    P = O.problem(O.FLUX_EULER1D, bc=O.BC_OUTFLOW, alpha_R=W.ALPHA_R_SEEDED)
    u_ref, du, _, s = O.run_jvp(P, U0[0], d, dx, cfl=CFL, n_steps=steps)
    assert s == steps
    assert np.array_equal(uT[0], u_ref)
    dj = dx * float(np.dot(u_ref[0] - target[0], du[0]))
    adj = float(np.sum(g0[0] * d))
    assert abs(adj - dj) <= 1e-9 * abs(dj), (adj, dj)


def test_adjoint_c5_shape_matches_dual_numbers(wtlib, oracle):
    """All 256 problems of the workload, strict mode, 256 RK steps (a bounded part of the 1024)
    with checkpoints every 32 (7 of 8 segments recomputed): on 64 seeded unit directions, one on
    each of problems 0..63, <g, d> equals the oracle's forward-mode (dual-number) derivative of
    the same map (OpenMP over the problems) to 1e-9 relative, and u(T) equals the oracle's bit for
    bit.  Central finite differences cannot stand in for the dual numbers at this size: on these
    data they differ from one another by 1e-3 to order one between h = 2.5e-7, 1e-6 and 4e-6
    (decisions on their thresholds and exactly tied maxima within the difference step, and the
    rounding of a loss whose variation is 1e-9 of its value), so the finite-difference checks use
    small smooth problems (test_gpu_adjoint.py)."""
    b, O = wtlib, oracle
    nprob, steps, ndir = 256, 256, 64
    U0, dx = W.adjoint_batch(nprob, N)
    Ut, _ = W.adjoint_batch(nprob, N, perturbed=True)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, mode=b.WT_MODE_STRICT, alpha_R=W.ALPHA_R_SEEDED)
    target = _forward(b, prob, Ut, steps)
    g0, uT = _adjoint(b, prob, U0, target, steps, dx)
    rng = np.random.default_rng(11)
    D = rng.standard_normal((ndir, 3, N))
    D /= np.linalg.norm(D.reshape(ndir, -1), axis=1)[:, None, None]
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    off = np.arange(ndir) * N
    u_ref, du = O.run_jvp_batch(P, U0[:ndir].transpose(1, 0, 2).reshape(3, -1), D.transpose(1, 0, 2).reshape(3, -1),
                                off, np.full(ndir, N), -5.0, 5.0, np.ones(ndir, np.int32), cfl=CFL, n_steps=steps)
    u_ref = u_ref.reshape(3, ndir, N).transpose(1, 0, 2)
    du = du.reshape(3, ndir, N).transpose(1, 0, 2)
    assert np.array_equal(uT[:ndir], u_ref)
    dj = dx * np.sum((u_ref[:, 0, :] - target[:ndir]) * du[:, 0, :], axis=1)
    adj = np.sum(g0[:ndir] * D, axis=(1, 2))
    rel = np.abs(adj - dj) / np.abs(dj)
    assert np.all(rel <= 1e-9), (rel.max(), int(np.argmax(rel)))

"""The wave-speed maxima of the stage tiles, at the edges of their FP32 screen.

The stage and batched tiles screen the wave speeds |u - c|, |u|, |u + c| of their output in
FP32 and take the FP64 speeds only of the cells that can hold a tile maximum.  The maxima
are the alpha_s of Eq. (flux_split_lf) for the next stage, so a cell missed by the screen
changes the result.  Each problem below puts the maxima where the screen is weakest: ties
below FP32 resolution, cells outside the range its error bound covers (internal energy under
E / 16, momenta under 2^-100, densities over 2^60), near-sonic flow (|u - c| cancelling), and
runs of bitwise-equal states.  Strict runs must equal the oracle bit for bit; fast batched
runs (stage tiles, screened) must equal fast single-problem runs of the same problems (the
step-blocked kernel, which takes every cell's FP64 speeds) bit for bit.
"""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")

N = 300
STEPS = 5


def _bump(n, c0, c1):
    """0 outside [c0, c1) (cell indices), a smooth bump of height 1 inside."""
    j = np.arange(n, dtype=np.float64)
    s = np.clip((j - c0) / max(c1 - c0, 1), 0.0, 1.0)
    return np.sin(np.pi * s) ** 2


def _problems():
    rng = np.random.default_rng(2024)
    r = lambda: rng.uniform(-1.0, 1.0, N)  # noqa: E731
    out = []
    # ties far below FP32 resolution
    out.append(W.cons_1d(1.0 + 1e-13 * r(), np.full(N, 0.3), np.ones(N)))
    out.append(W.cons_1d(1.0 + 1e-9 * r(), np.full(N, -0.7), 0.5 * (1.0 + 1e-9 * r())))
    # a high-Mach bump: internal energy below E / 16 (screen does not apply there)
    bm = _bump(N, 100, 160)
    out.append(W.cons_1d(np.ones(N), 0.5 + 3.5 * bm, 1.0 - 0.95 * bm))
    # momenta of 1e-35 (below 2^-100, not zero) beside exact zeros
    U = W.cons_1d(np.ones(N), np.zeros(N), np.ones(N))
    U[1, ::7] = 1e-35 * np.sign(r()[::7])
    out.append(U)
    # densities and pressures over 2^60 everywhere
    x = np.arange(N) / N
    out.append(W.cons_1d(2e18 * (1.0 + 0.1 * np.sin(6.0 * x)), np.full(N, 0.5), np.full(N, 2e18)))
    # internal energy at E / 16 up to 1e-7: kinetic = 15 x internal at p = 0.4, rho = 1
    out.append(W.cons_1d(np.ones(N), np.full(N, np.sqrt(30.0)), 0.4 * (1.0 + 1e-7 * r())))
    # near-sonic: u = c (1 + 1e-10 r), |u - c| cancels to 1e-10
    c = np.sqrt(1.4)
    out.append(W.cons_1d(np.ones(N), c * (1.0 + 1e-10 * r()), np.ones(N)))
    # exactly uniform, and uniform with one cell different (runs of equal states)
    out.append(W.cons_1d(np.full(N, 0.8), np.full(N, 0.25), np.full(N, 0.6)))
    U = W.cons_1d(np.full(N, 0.8), np.full(N, 0.25), np.full(N, 0.6))
    U[:, 151] = W.cons_1d([0.8], [0.2500000001], [0.6])[:, 0]
    out.append(U)
    return out


def _batch():
    probs = _problems()
    k = len(probs)
    lengths = np.full(k, N, dtype=np.int64)
    offsets = np.arange(k, dtype=np.int64) * N
    bc = np.array([p % 2 for p in range(k)], dtype=np.int32)  # periodic and outflow in turn
    return W.Batch(lengths, offsets, bc, np.full(k, 10.0 / N), np.full(k, -5.0), np.full(k, 5.0),
                   np.ascontiguousarray(np.concatenate(probs, axis=1)))


def _segments(b, batch):
    segs = []
    for p in range(len(batch.lengths)):
        s = b.WtSegment()
        s.offset, s.n = int(batch.offsets[p]), int(batch.lengths[p])
        s.lo, s.hi = float(batch.lo[p]), float(batch.hi[p])
        s.bc_lo = s.bc_hi = int(batch.bc[p])
        segs.append(s)
    return segs


def _run_batched(b, prob, batch, tile=None, monkeypatch=None):
    if tile is not None:
        monkeypatch.setenv("WT_BATCHED_TILE", str(tile))
    segs = _segments(b, batch)
    total = int(batch.u.shape[1])
    ws = b.alloc_workspace(b.workspace_bytes(prob, None, total, len(segs)))
    u = torch.from_numpy(batch.u.copy()).cuda()
    t = torch.zeros(len(segs), dtype=torch.float64, device="cuda")
    st = torch.zeros(len(segs), dtype=torch.int32, device="cuda")
    b.weno_theta_step_batched(prob, segs, u, total, 0.5, STEPS, ws, t_per_problem=t, status_per_problem=st)
    torch.cuda.synchronize()
    return u.cpu().numpy(), t.cpu().numpy(), st.cpu().numpy()


def test_screen_cases_are_what_they_claim():
    """The designed data reach the screen's edges: the high-Mach bump and the E / 16 problem
    hold cells on both sides of the internal-energy bound, the 1e-35 momenta lie in (0, 2^-100),
    the large problem lies above 2^60, and the near-sonic one has |u - c| <= 1e-9 c."""
    P = _problems()
    frac = lambda U: (U[2] - 0.5 * U[1] ** 2 / U[0]) / U[2]  # noqa: E731
    f = frac(P[2])
    assert (f < 1 / 16).any() and (f > 1 / 16).any()
    f = frac(P[5])
    assert (f < 1 / 16).any() and (f > 1 / 16).any()
    m = np.abs(P[3][1])
    assert ((m > 0) & (m < 2.0 ** -100)).sum() > 10 and (m == 0).sum() > 10
    assert (P[4][0] > 2.0 ** 60).all()
    rho, u = P[6][0], P[6][1] / P[6][0]
    c = np.sqrt(1.4 * 0.4 * (P[6][2] - 0.5 * rho * u * u) / rho)
    assert np.abs(u - c).max() <= 1e-9 * c.max()


@pytest.mark.gpu
def test_strict_batched_runs_equal_the_oracle(wtlib, oracle):
    b, O = wtlib, oracle
    batch = _batch()
    prob = b.problem(b.WT_FLUX_EULER1D, mode=b.WT_MODE_STRICT, alpha_R=W.ALPHA_R_SEEDED)
    u, t, st = _run_batched(b, prob, batch)
    for p in range(len(batch.lengths)):
        o = int(batch.offsets[p])
        P = O.problem(O.FLUX_EULER1D, bc=int(batch.bc[p]), alpha_R=W.ALPHA_R_SEEDED)
        ref, t_ref, s_ref = O.run(P, batch.u[:, o:o + N], float(batch.dx[p]), cfl=0.5, n_steps=STEPS)
        assert st[p] == 0 and s_ref == STEPS and t[p] == t_ref, (p, t[p], t_ref)
        assert np.array_equal(u[:, o:o + N], ref), (p, np.abs(u[:, o:o + N] - ref).max())


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [127, 5127])
def test_fast_batched_runs_equal_single_problem_runs(wtlib, monkeypatch, tile):
    b = wtlib
    batch = _batch()
    prob = b.problem(b.WT_FLUX_EULER1D, mode=b.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    u, t, st = _run_batched(b, prob, batch, tile, monkeypatch)
    for p in range(len(batch.lengths)):
        o = int(batch.offsets[p])
        pb = b.problem(b.WT_FLUX_EULER1D, bc=int(batch.bc[p]), mode=b.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
        g = b.grid_1d(N, -5.0, 5.0)
        ws = b.alloc_workspace(b.workspace_bytes(pb, g))
        us = torch.from_numpy(np.ascontiguousarray(batch.u[:, o:o + N])).cuda()
        ts, steps = b.weno_theta_step(pb, g, us, 0.5, ws, max_steps=STEPS)
        assert st[p] == 0 and steps == STEPS and ts == t[p], (p, ts, t[p])
        assert np.array_equal(us.cpu().numpy(), u[:, o:o + N]), p

"""Batched stepping (many independent 1D problems in one launch per RK stage) against the
oracle, problem by problem, and against single-problem GPU runs."""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHOCK_L1_TOL = 1e-10


def _segments(b, batch):
    segs = []
    for p in range(len(batch.lengths)):
        s = b.WtSegment()
        s.offset = int(batch.offsets[p])
        s.n = int(batch.lengths[p])
        s.lo, s.hi = float(batch.lo[p]), float(batch.hi[p])
        bc = int(batch.bc[p])
        s.bc_lo = s.bc_hi = bc
        segs.append(s)
    return segs


def _run_batched(b, prob, batch, n_steps, cfl=0.5, host=False):
    segs = _segments(b, batch)
    total = int(batch.u.shape[1])
    ws = b.alloc_workspace(b.workspace_bytes(prob, None, total, len(segs)))
    if host:
        u = np.ascontiguousarray(batch.u).copy()
        t = np.zeros(len(segs))
        b.weno_theta_step_batched(prob, segs, u, total, cfl, n_steps, ws, t_per_problem=t)
        return u, t
    u = torch.from_numpy(np.ascontiguousarray(batch.u)).cuda()
    t = torch.zeros(len(segs), dtype=torch.float64, device="cuda")
    b.weno_theta_step_batched(prob, segs, u, total, cfl, n_steps, ws, t_per_problem=t)
    torch.cuda.synchronize()
    return u.cpu().numpy(), t.cpu().numpy()


def _oracle_one(O, batch, p, n_steps, cfl=0.5, flux=None):
    o, n = int(batch.offsets[p]), int(batch.lengths[p])
    U = batch.u[:, o:o + n]
    P = O.problem(O.FLUX_EULER1D if flux is None else flux, bc=int(batch.bc[p]),
                  alpha_R=W.ALPHA_R_SEEDED if flux is None else 50.0)
    return O.run(P, U, float(batch.dx[p]), cfl=cfl, n_steps=n_steps)


EDGE_LENGTHS = [3, 4, 5, 31, 32, 33, 62, 63, 64, 126, 127, 128, 129, 255, 700, 1500]


def test_batched_strict_matches_oracle_problem_by_problem(wtlib, oracle):
    b, O = wtlib, oracle
    batch = W.euler_batch(len(EDGE_LENGTHS), seed=4, lengths=EDGE_LENGTHS)
    prob = b.problem(b.WT_FLUX_EULER1D, mode=b.WT_MODE_STRICT, alpha_R=W.ALPHA_R_SEEDED)
    u, t = _run_batched(b, prob, batch, 15)
    for p in range(len(EDGE_LENGTHS)):
        ref, t_ref, s_ref = _oracle_one(O, batch, p, 15)
        o, n = int(batch.offsets[p]), int(batch.lengths[p])
        assert s_ref == 15 and t[p] == t_ref, (p, t[p], t_ref)
        assert np.array_equal(u[:, o:o + n], ref), (p, n, np.abs(u[:, o:o + n] - ref).max())


def test_batched_fast_equals_single_problem_runs(wtlib):
    b = wtlib
    batch = W.euler_batch(24, seed=9, nmin=64, nmax=4000)
    prob = b.problem(b.WT_FLUX_EULER1D, mode=b.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    u, t = _run_batched(b, prob, batch, 12)
    for p in range(24):
        o, n = int(batch.offsets[p]), int(batch.lengths[p])
        pb = b.problem(b.WT_FLUX_EULER1D, bc=int(batch.bc[p]), mode=b.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
        g = b.grid_1d(n, -5.0, 5.0)
        ws = b.alloc_workspace(b.workspace_bytes(pb, g))
        us = torch.from_numpy(np.ascontiguousarray(batch.u[:, o:o + n])).cuda()
        ts, steps = b.weno_theta_step(pb, g, us, 0.5, ws, max_steps=12)
        assert steps == 12 and ts == t[p]
        assert np.array_equal(us.cpu().numpy(), u[:, o:o + n]), p


def test_batched_scalar_strict_and_host_arrays(wtlib, oracle):
    b, O = wtlib, oracle
    lengths = [3, 40, 64, 65, 200, 333]
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    rng = np.random.default_rng(3)
    u = np.zeros((1, sum(lengths)))
    dx = []
    for p, n in enumerate(lengths):
        x, d = W.grid_1d(n, -1.0, 1.0, periodic=True)
        u[0, offsets[p]:offsets[p] + n] = np.sin(np.pi * x + rng.uniform(0, 6)) + 0.5 * (x > rng.uniform(-0.5, 0.5))
        dx.append(d)
    batch = W.Batch(np.array(lengths), offsets, np.zeros(len(lengths), np.int32), np.array(dx),
                    np.full(len(lengths), -1.0), np.full(len(lengths), 1.0), u)
    for flux in (b.WT_FLUX_ADVECTION, b.WT_FLUX_BURGERS):
        prob = b.problem(flux, mode=b.WT_MODE_STRICT)
        ud, td = _run_batched(b, prob, batch, 10, cfl=0.4)
        uh, th = _run_batched(b, prob, batch, 10, cfl=0.4, host=True)
        assert np.array_equal(ud, uh) and np.array_equal(td, th)
        for p, n in enumerate(lengths):
            ref, t_ref, _ = _oracle_one(O, batch, p, 10, cfl=0.4, flux=flux)
            assert np.array_equal(ud[:, offsets[p]:offsets[p] + n], ref), (flux, p)
            assert td[p] == t_ref


def test_batched_full_size_sampled(wtlib, oracle):
    """The batched workload at full size (4096 problems, lengths log-uniform in [256, 65536],
    mixed periodic/outflow, per-problem CFL step), as the benchmark launches it (fast mode),
    for a bounded number of RK steps; sampled problems are recomputed by the oracle."""
    b, O = wtlib, oracle
    steps = 20
    batch = W.euler_batch(4096, seed=0)
    prob = b.problem(b.WT_FLUX_EULER1D, mode=b.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    u, t = _run_batched(b, prob, batch, steps)
    order = np.argsort(batch.lengths)
    sample = [int(order[0]), int(order[1]), int(order[2048]), int(order[-2]), int(order[-1])]
    sample += [1301, 1994]  # problems whose stages pass through negative pressure / break down with alpha_R = 50
    sample += [int(i) for i in np.random.default_rng(1).choice(4096, 5, replace=False)]
    for p in sample:
        ref, t_ref, _ = _oracle_one(O, batch, p, steps)
        o, n = int(batch.offsets[p]), int(batch.lengths[p])
        assert abs(t[p] - t_ref) <= 1e-13 * t_ref
        l1 = batch.dx[p] * np.abs(u[:, o:o + n] - ref).sum(axis=1)
        assert np.all(l1 <= SHOCK_L1_TOL), (p, n, l1)

"""The oracle's batch runner (OpenMP over independent problems, used for the all-core CPU
baseline and for full-length parity on large batches) is the serial single-problem run,
problem by problem, bit for bit, whatever the thread count."""
import numpy as np

from paper_1504_00731_gb300 import workloads as W


def test_run_batch_equals_single_problem_runs(oracle):
    O = oracle
    b = W.euler_batch(10, seed=4, nmin=8, nmax=96)
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    one, s1 = O.run_batch(P, b.u, b.offsets, b.lengths, b.lo, b.hi, b.bc, cfl=0.5, n_steps=4, threads=1)
    many, s2 = O.run_batch(P, b.u, b.offsets, b.lengths, b.lo, b.hi, b.bc, cfl=0.5, n_steps=4, threads=0)
    assert np.array_equal(one, many) and np.array_equal(s1, s2) and (s1 == 4).all()
    for p in range(10):
        o, n = int(b.offsets[p]), int(b.lengths[p])
        Q = O.problem(O.FLUX_EULER1D, bc=int(b.bc[p]), alpha_R=W.ALPHA_R_SEEDED)
        ref, _, steps = O.run(Q, b.u[:, o:o + n], b.dx[p], cfl=0.5, n_steps=4)
        assert steps == 4
        assert np.array_equal(one[:, o:o + n], ref)
    assert O.max_threads() >= 1


def test_run_jvp_batch_equals_single_problem_runs(oracle):
    O = oracle
    b = W.euler_batch(6, seed=5, nmin=8, nmax=64)
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    d = np.random.default_rng(2).standard_normal(b.u.shape)
    u, du = O.run_jvp_batch(P, b.u, d, b.offsets, b.lengths, b.lo, b.hi, b.bc, cfl=0.5, n_steps=3)
    for p in range(6):
        o, n = int(b.offsets[p]), int(b.lengths[p])
        Q = O.problem(O.FLUX_EULER1D, bc=int(b.bc[p]), alpha_R=W.ALPHA_R_SEEDED)
        ru, rdu, _, _ = O.run_jvp(Q, b.u[:, o:o + n], d[:, o:o + n], b.dx[p], cfl=0.5, n_steps=3)
        assert np.array_equal(u[:, o:o + n], ru) and np.array_equal(du[:, o:o + n], rdu)

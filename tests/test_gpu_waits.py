"""Failure detection without a GPU fault: every device-side wait in the kernels is bounded, and
a wait that can never be satisfied gives up and reports WT_ERR_TIMEOUT through the status the
host reads, leaving the context usable.  The waits run out on purpose here (a grid counter no
block increments, an mbarrier whose bulk-copy bytes are never sent, mailbox words that never
take the awaited tag or parity); nothing is left in flight and nothing traps."""
import numpy as np
import pytest

from paper_1504_00731_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_unsatisfiable_waits_time_out_and_the_context_survives(wtlib):
    b = wtlib
    ws = b.alloc_workspace(256)
    limit = 1 << 20  # about half a millisecond of SM clock
    assert b.selftest_wait(0, limit, ws) == b.WT_ERR_TIMEOUT
    assert "gave up" in b.last_error()
    assert b.selftest_wait(1, limit, ws) == b.WT_ERR_TIMEOUT
    assert b.selftest_wait(2, limit, ws) == b.WT_OK
    # the step-blocked kernel's mailboxes: halo words whose tag never comes, alpha words that
    # never take the step's parity, and alpha words already published
    assert b.selftest_wait(3, limit, ws) == b.WT_ERR_TIMEOUT
    assert b.selftest_wait(4, limit, ws) == b.WT_ERR_TIMEOUT
    assert b.selftest_wait(5, limit, ws) == b.WT_OK
    # the context is still usable: a step runs and matches a fresh run
    U, x, dx = W.euler_c2(512, seed=4)
    prob = b.problem(b.WT_FLUX_EULER1D, bc=b.WT_BC_OUTFLOW, alpha_R=W.ALPHA_R_SEEDED)
    g = b.grid_1d(512, -5.0, 5.0)
    w = b.alloc_workspace(b.workspace_bytes(prob, g))
    u = torch.from_numpy(U).cuda()
    t, s = b.weno_theta_step(prob, g, u, 0.5, w, max_steps=20)
    assert s == 20 and bool(torch.isfinite(u).all())

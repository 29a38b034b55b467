"""Two gloo ranks on the CPU run the multi-GPU host logic: each rank advances its own seeded
problem (here with the oracle, no GPU), timings reduce to the maximum, and the whole-job rate
counts every rank's work."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import time

    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1504_00731_gb300 import distributed as D
    from paper_1504_00731_gb300 import workloads as W
    import oracle as O

    w, r, lr = D.env()
    seed = D.rank_seed(0, r)
    U, x, dx = W.euler_c2(256, seed=seed)
    t0 = time.perf_counter()
    u, t, steps = O.run(O.problem(O.FLUX_EULER1D, bc=O.BC_OUTFLOW, alpha_R=W.ALPHA_R_SEEDED), U, dx, cfl=0.5,
                        n_steps=5)
    el = time.perf_counter() - t0 + 0.01 * r  # rank 1 deliberately slower
    mx = D.max_over_ranks(el)
    rate = D.whole_job_rate(256 * 5, w, mx)
    out.put((r, w, seed, float(u.sum()), el, mx, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_independent_problems():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, w0, s0, sum0, el0, mx0, rate0), (r1, w1, s1, sum1, el1, mx1, rate1) = res
    assert (w0, w1) == (2, 2) and s0 != s1 and sum0 != sum1  # different seeded problems
    assert mx0 == mx1 == pytest.approx(max(el0, el1))        # max over ranks
    assert rate0 == rate1 == pytest.approx(2 * 256 * 5 / max(el0, el1))

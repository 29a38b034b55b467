"""The multi-GPU host logic on two gloo ranks (CPU, no GPU): the batched workload is split by
problem with the LPT partition, each rank advances its share (here with the oracle), and the
shares put back together equal a single-rank run of the whole batch bit for bit.  Timings
reduce to the maximum over ranks, and the whole-job rate counts every rank's cells."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1504_00731_gb300 import distributed as D

NPROB, NMIN, NMAX, STEPS = 24, 16, 160, 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_lpt_partition_properties():
    """Every problem on exactly one rank; the ranks' cell totals within the largest problem of
    each other (the LPT bound for a partition on lengths); deterministic."""
    from paper_1504_00731_gb300 import workloads as W

    for world in (1, 2, 3, 8):
        lengths = W.batch_lengths(4096, seed=0)
        parts = D.lpt_partition(lengths, world)
        assert len(parts) == world
        allp = np.concatenate(parts)
        assert np.array_equal(np.sort(allp), np.arange(len(lengths)))
        loads = np.array([lengths[p].sum() for p in parts])
        assert loads.max() - loads.min() <= lengths.max()
        again = D.lpt_partition(lengths, world)
        assert all(np.array_equal(a, b) for a, b in zip(parts, again))
    # a hand-checked case: 7, 5, 4, 3, 1 on two ranks: 7 -> r0, 5 -> r1, 4 -> r1 (9),
    # 3 -> r0 (10), 1 -> r1 (10)
    parts = D.lpt_partition([3, 7, 1, 5, 4], 2)
    assert [list(p) for p in parts] == [[1, 0], [3, 4, 2]]


def _worker(rank, world, port, out):
    import time

    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1504_00731_gb300 import workloads as W
    import oracle as O

    w, r, lr = D.env()
    lengths = W.batch_lengths(NPROB, seed=3, nmin=NMIN, nmax=NMAX)
    mine = D.lpt_partition(lengths, w)[r]
    b = W.euler_batch(NPROB, seed=3, nmin=NMIN, nmax=NMAX, problems=mine)
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    t0 = time.perf_counter()
    u, steps = O.run_batch(P, b.u, b.offsets, b.lengths, b.lo, b.hi, b.bc, cfl=0.5, n_steps=STEPS, threads=1)
    el = time.perf_counter() - t0 + 0.01 * r  # rank 1 deliberately slower
    mx = D.max_over_ranks(el)
    cells = D.sum_over_ranks(float(b.lengths.sum()))
    rate = D.whole_job_rate(cells * STEPS, mx)
    out.put((r, w, mine.tolist(), u, el, mx, cells, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_by_lpt():
    from paper_1504_00731_gb300 import workloads as W
    import oracle as O

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
    res.sort(key=lambda x: x[0])
    whole = W.euler_batch(NPROB, seed=3, nmin=NMIN, nmax=NMAX)
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    ref, _ = O.run_batch(P, whole.u, whole.offsets, whole.lengths, whole.lo, whole.hi, whole.bc, cfl=0.5,
                         n_steps=STEPS, threads=1)
    seen = []
    for r, w, mine, u, el, mx, cells, rate in res:
        assert w == 2
        o = 0
        for p in mine:  # the rank's share is packed in its own order
            n = int(whole.lengths[p])
            a, b = int(whole.offsets[p]), int(whole.offsets[p]) + n
            assert np.array_equal(u[:, o:o + n], ref[:, a:b]), p
            o += n
            seen.append(p)
    assert sorted(seen) == list(range(NPROB))
    loads = [sum(int(whole.lengths[p]) for p in x[2]) for x in res]
    assert abs(loads[0] - loads[1]) <= int(whole.lengths.max())
    els = [x[4] for x in res]
    for x in res:
        assert x[5] == pytest.approx(max(els))                     # max over ranks
        assert x[6] == float(whole.lengths.sum())                   # cells of all ranks
        assert x[7] == pytest.approx(whole.lengths.sum() * STEPS / max(els))


def test_batch_prefix_is_the_single_gpu_batch():
    """The N-rank workload is the first N x 4096 problems of the seed-0 stream, whose first 4096
    are exactly the single-GPU batch (lengths, boundaries and data)."""
    from paper_1504_00731_gb300 import workloads as W

    a = W.batch_lengths(64, seed=0)
    b = W.batch_lengths(128, seed=0)
    assert np.array_equal(a, b[:64])
    x = W.euler_batch(8, seed=0, nmin=16, nmax=64)
    y = W.euler_batch(16, seed=0, nmin=16, nmax=64, problems=np.arange(8))
    assert np.array_equal(x.u, y.u) and np.array_equal(x.bc, y.bc)

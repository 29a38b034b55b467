"""The algorithmic flop counts bench.py divides by are the oracle's operation counts."""
import re

from paper_1504_00731_gb300 import workloads as W


def _bench_constant(name):
    src = open(__file__.replace("tests/test_flop_count.py", "bench.py")).read()
    return float(re.search(rf"^{name} = ([0-9.]+)", src, re.M).group(1))


def test_bench_flop_constants_match_the_oracle_count(oracle):
    O = oracle
    U, x, dx = W.euler_c2(4096, seed=0)
    c = O.count_run_ops(O.problem(O.FLUX_EULER1D, bc=O.BC_OUTFLOW, alpha_R=W.ALPHA_R_SEEDED), U, dx, cfl=0.5, n_steps=1)
    per = (c["add"] + c["mul"] + c["div"] + c["sqrt"]) / 4096
    assert abs(per - _bench_constant("FLOPS_PER_CELL_UPDATE")) < 1.0
    U2, dx2, dy2 = W.euler2d_vortices(64, 64, seed=0)
    c = O.count_run_ops(O.problem(O.FLUX_EULER2D, bc=O.BC_PERIODIC, alpha_R=W.ALPHA_R_SEEDED), U2, dx2, dy2,
                        cfl=0.45, n_steps=1)
    per2 = (c["add"] + c["mul"] + c["div"] + c["sqrt"]) / 64 / 64
    assert abs(per2 - _bench_constant("FLOPS_PER_CELL_UPDATE_2D")) < 2.0

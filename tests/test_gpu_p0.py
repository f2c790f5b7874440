"""GPU parity of P0-DG (LMDG_P0: S_N-DG on the piecewise constants, Section 3.1's comparison scheme) against the
oracle's L00 sweeps: operator applications and source residuals at 1e-12, FP32 sweeps at 1e-5, solves at 1e-10
of the oracle's direct solve, and the 1024^2 S16 benchmark medium."""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import random_problem, rel
from workloads.problems import config4

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,N,eps,seed", [(1, 4, 1.0, 1), (5, 4, 1.0, 2), (37, 4, 1e-2, 3), (40, 8, 1.0, 5),
                                          (70, 4, 0.3, 4)])
def test_operator_apply(n, N, eps, seed):
    from paper_1907_01027_gb300 import Context, SWEEP_FP32, SWEEP_SOURCE
    p = random_problem(n, N, eps, seed)
    so = SweepOracle(p)
    ctx = Context(p, "p0")
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    ref = so.K("p0", x)
    assert rel(y, ref) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_SOURCE), ref - so.rhs("p0")) < 1e-12
    if eps == 1.0:
        assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    ctx.close()


@pytest.mark.parametrize("n,N,eps,seed", [(9, 4, 1.0, 21), (16, 4, 0.1, 22), (12, 8, 1.0, 23)])
def test_solve_matches_oracle(n, N, eps, seed):
    from paper_1907_01027_gb300 import Context
    p = random_problem(n, N, eps, seed)
    ref = SweepOracle(p).solve("p0", direct=True)
    ctx = Context(p, "p0", tol=1e-13, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0, st
    assert rel(phi, ref["phi"]) < 1e-10
    assert rel(ctx.get_psi(), ref["psi0"]) < 1e-10
    ctx.close()


def test_operator_apply_1024_s16():
    from paper_1907_01027_gb300 import Context, SWEEP_FP32
    p = config4(eps=1.0)
    ctx = Context(p, "p0")
    x = np.random.default_rng(7).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    assert rel(y, SweepOracle(p).K("p0", x)) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    ctx.close()

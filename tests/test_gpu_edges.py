"""Degenerate and ragged sizes against the oracle: a single cell, meshes around one and two 32-row strips and
ragged last strips, the smallest quadrature (S2, four directions), vacuum and inflow data."""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import random_problem, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("n,N", [(1, 2), (1, 4), (2, 2), (3, 2), (16, 4), (31, 4), (32, 2), (33, 4), (63, 2),
                                 (64, 2), (65, 2), (97, 2)])
def test_edge_sizes(variant, n, N):
    from paper_1907_01027_gb300 import Context, SWEEP_SOURCE, SWEEP_FP32
    p = random_problem(n, N, 0.5, 200 + n + N)
    so = SweepOracle(p)
    ctx = Context(p, variant)
    x = np.random.default_rng(n).standard_normal((p.nx, 4))
    ref = so.K(variant, x)
    assert rel(ctx.sweep(x), ref) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_FP32), ref) < 1e-5
    if 4 * p.nx <= 1024:                      # the oracle solves these directly (no iteration error)
        ctx2 = Context(p, variant, tol=1e-13, max_iters=20000)
        _, phi, st, rc = ctx2.solve()
        assert rc == 0
        assert rel(phi, so.solve(variant, direct=True)["phi"]) < 1e-9
        ctx2.close()
    ctx.close()

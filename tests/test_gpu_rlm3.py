"""GPU parity of RLMDG* (RLMDG with the three-cell reconstruction, lmdg_options.recon = 1) against the oracle's
sweeps with the same reading.  Meshes from 2 cells per side (no third cell) to ragged multi-strip sizes, and
the 1024^2 S16 benchmark pattern in optically thick cells; tolerances as for the other schemes (FP64 1e-12,
solves 1e-10 of the oracle's direct solve, FP32 sweeps 1e-5 of FP64 at eps = 1).
"""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import random_problem, rel
from workloads.problems import config4

pytestmark = pytest.mark.gpu


def _bprime(so):
    b = so.rhs("rlm")
    e = np.zeros((so.nx, 4))
    e[:, 1:] = so._rlm_F()[1]
    return b - so.K("rlm", e)


@pytest.mark.parametrize("n,N,eps,seed", [(2, 4, 1.0, 1), (5, 4, 1.0, 2), (37, 4, 1e-2, 3), (40, 8, 1.0, 5),
                                          (70, 4, 0.3, 4)])
def test_operator_apply(n, N, eps, seed):
    from paper_1907_01027_gb300 import Context, SWEEP_FP32, SWEEP_SOURCE
    p = random_problem(n, N, eps, seed)
    so = SweepOracle(p, three_cell=True)
    ctx = Context(p, "rlm", recon=1)
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    ref = so.K("rlm", x)
    assert rel(y, ref) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_SOURCE), ref - _bprime(so)) < 1e-12
    if eps == 1.0:
        assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    if n > 2:
        plain = Context(p, "rlm")
        assert rel(plain.sweep(x), y) > 1e-8
        plain.close()
    ctx.close()


@pytest.mark.parametrize("n,N,eps,seed", [(9, 4, 1.0, 21), (16, 4, 0.1, 22), (12, 8, 1.0, 23)])
def test_solve_matches_oracle(n, N, eps, seed):
    from paper_1907_01027_gb300 import Context
    p = random_problem(n, N, eps, seed)
    ref = SweepOracle(p, three_cell=True).solve("rlm", direct=True)
    ctx = Context(p, "rlm", recon=1, tol=1e-13, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0, st
    assert rel(phi, ref["phi"]) < 1e-10
    assert rel(ctx.get_psi(), ref["psi0"]) < 1e-10
    ctx.close()


def test_operator_apply_1024_s16():
    # the benchmark's patch pattern with cross sections x1000 (sigma_t h from 0.2 to 20): in optically thin cells
    # the three-cell sweep amplifies round-off along a ray (pinned in the oracle tests), so parity at 1e-12 is
    # only defined where the scheme is stable
    from paper_1907_01027_gb300 import Context, SWEEP_FP32
    p = config4(eps=1.0)
    p.sigma_s = p.sigma_s * 1000.0
    p.sigma_a = p.sigma_a * 1000.0
    ctx = Context(p, "rlm", recon=1)
    x = np.random.default_rng(7).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    assert rel(y, SweepOracle(p, literal_b11=True, three_cell=True).K("rlm", x)) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    ctx.close()

"""GPU parity of RLMDG with the reconstruction suppressed across cross-section jumps (the remedy Section 4 gives
for the kinks at a discontinuity) against the oracle's sweeps with the same reading.

Media: two materials on random square patches, so that jumps cross x- and y-faces, strip boundaries and the
ragged last strip.  Tolerances as for the other schemes: FP64 applications 1e-12, solves 1e-10 of the
oracle's direct solve, FP32 sweeps 1e-5 of FP64 at eps = 1.
"""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import random_problem, rel
from workloads.problems import config4

pytestmark = pytest.mark.gpu


def _two_material(n, N, eps, seed, patch):
    p = random_problem(n, N, eps, seed)
    rng = np.random.default_rng(seed + 50)
    k = -(-n // patch)
    m = np.kron(rng.integers(0, 2, (k, k)), np.ones((patch, patch), dtype=int))[:n, :n].ravel()
    p.sigma_s = np.where(m == 1, 2.0, 0.7)
    p.sigma_a = np.where(m == 1, 0.3, 1.1)
    return p


def _bprime(so):
    b = so.rhs("rlm")
    e = np.zeros((so.nx, 4))
    e[:, 1:] = so._rlm_F()[1]
    return b - so.K("rlm", e)


@pytest.mark.parametrize("n,N,eps,seed,patch", [(5, 4, 1.0, 1, 1), (37, 4, 1.0, 2, 3), (37, 4, 1e-2, 3, 2),
                                                (40, 8, 1.0, 5, 4), (70, 4, 0.3, 4, 7)])
def test_operator_apply(n, N, eps, seed, patch):
    from paper_1907_01027_gb300 import Context, SWEEP_FP32, SWEEP_SOURCE
    p = _two_material(n, N, eps, seed, patch)
    so = SweepOracle(p, suppress=True)
    ctx = Context(p, "rlm", suppress=1)
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    ref = so.K("rlm", x)
    assert rel(y, ref) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_SOURCE), ref - _bprime(so)) < 1e-12
    if eps == 1.0:
        assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    # the plain scheme differs on this medium
    plain = Context(p, "rlm")
    assert rel(plain.sweep(x), y) > 1e-8
    plain.close()
    ctx.close()


@pytest.mark.parametrize("n,N,eps,seed", [(9, 4, 1.0, 21), (16, 4, 0.1, 22), (12, 8, 1.0, 23)])
def test_solve_matches_oracle(n, N, eps, seed):
    from paper_1907_01027_gb300 import Context
    p = _two_material(n, N, eps, seed, 3)
    ref = SweepOracle(p, suppress=True).solve("rlm", direct=True)
    ctx = Context(p, "rlm", suppress=1, tol=1e-13, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0, st
    assert rel(phi, ref["phi"]) < 1e-10
    assert rel(ctx.get_psi(), ref["psi0"]) < 1e-10
    ctx.close()


def test_homogeneous_medium_bitwise_plain():
    from paper_1907_01027_gb300 import Context
    p = random_problem(40, 4, 1.0, 31)
    p.sigma_s[:] = 1.1
    p.sigma_a[:] = 0.6
    x = np.random.default_rng(3).standard_normal((p.nx, 4))
    a, b = Context(p, "rlm"), Context(p, "rlm", suppress=1)
    assert np.array_equal(a.sweep(x), b.sweep(x))
    a.close()
    b.close()


def test_operator_apply_1024_s16():
    # the benchmark medium: 16x16-cell patches of distinct cross sections, jumps on every patch boundary
    from paper_1907_01027_gb300 import Context, SWEEP_FP32
    p = config4(eps=1.0)
    ctx = Context(p, "rlm", suppress=1)
    x = np.random.default_rng(7).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    assert rel(y, SweepOracle(p, literal_b11=True, suppress=True).K("rlm", x)) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    ctx.close()

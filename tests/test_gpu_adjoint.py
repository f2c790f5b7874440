"""GPU adjoint (lmdg_adjoint, standard scheme) against the oracle and against finite differences."""
import copy

import numpy as np
import pytest

from oracle.sweeps import SweepOracle, adjoint_std
from tests.helpers import random_problem, rel
from workloads.problems import config5

pytestmark = pytest.mark.gpu


def _ctx(p, **kw):
    from paper_1907_01027_gb300 import Context
    return Context(p, "std", **kw)


def test_adjoint_matches_oracle():
    p = random_problem(12, 8, 0.6, 91, q_per_angle=False)
    g = np.random.default_rng(92).uniform(0, 1, p.nx)
    J0, a0, b0, c0, _, _ = adjoint_std(SweepOracle(p), g, direct=True)
    ctx = _ctx(p, tol=1e-13, max_iters=20000)
    J, dss, dsa, dq, st = ctx.adjoint(g)
    assert abs(J - J0) <= 1e-10 * abs(J0)
    assert rel(dss, a0) < 1e-9 and rel(dsa, b0) < 1e-9 and rel(dq, c0) < 1e-9
    ctx.close()


def _J(p, g):
    ctx = _ctx(p, tol=1e-13, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    ctx.close()
    assert rc == 0
    return float(np.sum(g * p.h * p.h * phi[:, 0]))


def test_adjoint_finite_differences_bump_medium():
    # the adjoint workload's medium (sigma_s = 1 + 8 Gaussian bumps, sigma_a = 0.1, detector x > 0.9) on 32^2, S8
    p = config5(n=32)
    g = p.info["detector"]
    ctx = _ctx(p, tol=1e-13, max_iters=20000)
    J, dss, dsa, dq, st = ctx.adjoint(g)
    ctx.close()
    cells = np.random.default_rng(1908).choice(p.nx, 6, replace=False)
    for K in cells:
        for field, ref in (("sigma_s", dss), ("sigma_a", dsa)):
            d = 1e-3 * getattr(p, field)[K]
            pp, pm = copy.deepcopy(p), copy.deepcopy(p)
            getattr(pp, field)[K] += d
            getattr(pm, field)[K] -= d
            fd = (_J(pp, g) - _J(pm, g)) / (2 * d)
            assert abs(fd - ref[K]) <= 1e-6 * abs(ref[K]) + 1e-12 * abs(J), (field, K, fd, ref[K])
        pq = copy.deepcopy(p)
        pq.q[K, 0] += 1.0
        assert abs((_J(pq, g) - J) - dq[K]) <= 1e-9 * abs(J), (K, _J(pq, g) - J, dq[K])


def test_mixed_precision_adjoint_close_to_fp64():
    p = config5(n=32)
    g = p.info["detector"]
    c64 = _ctx(p, tol=1e-12)
    ref = c64.adjoint(g)
    c64.close()
    c32 = _ctx(p, tol=1e-12, precision=1)
    out = c32.adjoint(g)
    c32.close()
    assert abs(out[0] - ref[0]) <= 1e-10 * abs(ref[0])
    for i in (1, 2, 3):
        assert rel(out[i], ref[i]) < 1e-5


def test_lowmem_adjoint_matches_dense_oracle():
    from oracle import dense
    from paper_1907_01027_gb300 import Context
    p = random_problem(4, 4, 0.6, 93, q_per_angle=False)
    g = np.random.default_rng(94).uniform(0, 1, p.nx)
    J0, a0, b0, c0 = dense.adjoint(p, g, "lm")
    ctx = Context(p, "lm", tol=1e-13, max_iters=20000)
    J, dss, dsa, dq, st = ctx.adjoint(g)
    ctx.close()
    assert abs(J - J0) <= 1e-10 * abs(J0)
    assert rel(dss, a0) < 1e-9 and rel(dsa, b0) < 1e-9 and rel(dq, c0) < 1e-9

"""GPU parity of RLMDG with the Q1-type reconstruction (lmdg_options.recon = 2: the two-cell P1 slopes plus the
xi eta coefficient from the upwind y-difference of the reconstructed x-slopes) against the oracle's sweeps with the
same reading: operator applications (homogeneous and with source and inflow data, FP64 1e-12, float-float 3e-11,
FP32 1e-5 at eps = 1) on square, rectangular and multi-strip meshes, solves against the oracle's direct solve, and
the anisotropic bilinear state the reconstruction reproduces exactly.
"""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import random_problem, rel
from workloads.problems import mms_problem

pytestmark = pytest.mark.gpu


def _bprime(so):
    b = so.rhs("rlm")
    e = np.zeros((so.nx, 4))
    e[:, 1:] = so._rlm_F()[1]
    return b - so.K("rlm", e)


@pytest.mark.parametrize("n,ny,N,eps,seed", [(2, 0, 4, 1.0, 1), (5, 0, 4, 1.0, 2), (37, 0, 4, 1e-2, 3),
                                             (40, 20, 8, 1.0, 5), (20, 45, 4, 0.5, 6), (70, 0, 4, 0.3, 4)])
def test_operator_apply(n, ny, N, eps, seed):
    from paper_1907_01027_gb300 import Context, SWEEP_FP32, SWEEP_SOURCE, SWEEP_F32X2
    p = random_problem(n, N, eps, seed, ny=ny)
    so = SweepOracle(p, q1=True)
    ctx = Context(p, "rlm", recon=2)
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    ref = so.K("rlm", x)
    assert rel(y, ref) < 1e-12
    refs = ref - _bprime(so)
    assert rel(ctx.sweep(x, flags=SWEEP_SOURCE), refs) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_SOURCE | SWEEP_F32X2), refs) < 3e-11
    if eps == 1.0:
        assert rel(ctx.sweep(x, flags=SWEEP_FP32), y) < 1e-5
    plain = Context(p, "rlm")
    assert rel(plain.sweep(x)[:, 0], y[:, 0]) < 1e-12          # the cell-average rows are RLMDG's
    assert rel(plain.sweep(x), y) > 1e-8                       # the slope rows are not
    plain.close()
    ctx.close()


@pytest.mark.parametrize("n,N,eps,seed", [(9, 4, 1.0, 21), (12, 8, 1.0, 23)])
def test_solve_matches_oracle(n, N, eps, seed):
    from paper_1907_01027_gb300 import Context
    p = random_problem(n, N, eps, seed)
    ref = SweepOracle(p, q1=True).solve("rlm", direct=True)
    ctx = Context(p, "rlm", recon=2, tol=1e-13, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0, st
    assert rel(phi, ref["phi"]) < 1e-10
    assert rel(ctx.get_psi(), ref["psi0"]) < 1e-10
    ctx.close()


def test_anisotropic_bilinear_state_exact():
    """psi_l = (Omega_x - 2 Omega_y)^2 x y + 0.3: the Q1-type scheme's cell averages are exact to round-off on the
    GPU, two-cell RLMDG's are not."""
    from paper_1907_01027_gb300 import Context
    c = lambda a, b: (a - 2 * b) ** 2
    p = mms_problem(24, 4, lambda x, y, a, b: c(a, b) * x * y + 0.3, lambda x, y, a, b: c(a, b) * y,
                    lambda x, y, a, b: c(a, b) * x, sigma_s=1.3, sigma_a=0.4, eps=0.7)
    exact = p.info["phi_avg"]
    ctx = Context(p, "rlm", recon=2, tol=1e-13, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    ctx.close()
    assert rc == 0 and np.abs(phi[:, 0] - exact).max() < 1e-10, st
    two = Context(p, "rlm", tol=1e-13, max_iters=20000)
    _, phi2, _, _ = two.solve()
    two.close()
    assert np.abs(phi2[:, 0] - exact).max() > 1e-7

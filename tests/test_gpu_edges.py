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


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("nx,ny,N", [(37, 70, 4), (70, 37, 2), (1, 65, 2), (65, 1, 4), (2, 33, 2), (33, 2, 2),
                                     (5, 3, 4)])
def test_rectangular_meshes(variant, nx, ny, N):
    """nx x ny meshes (Section 2.1's Cartesian mesh need not be square): one and several 32-row strips with
    ragged last strips, single rows and columns; operator parity 1e-12 and, where the oracle solves directly,
    the solution and the stored angular unknowns."""
    from paper_1907_01027_gb300 import Context, SWEEP_FP32, SWEEP_SOURCE
    p = random_problem(nx, N, 0.5, 300 + nx + 3 * ny, ny=ny)
    so = SweepOracle(p)
    ctx = Context(p, variant)
    x = np.random.default_rng(nx * ny).standard_normal((p.nx, 4))
    ref = so.K(variant, x)
    assert rel(ctx.sweep(x), ref) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_FP32), ref) < 1e-5
    ctx.close()
    if 4 * p.nx <= 600:
        ctx2 = Context(p, variant, tol=1e-13, max_iters=20000)
        _, phi, st, rc = ctx2.solve()
        assert rc == 0
        d = so.solve(variant, direct=True)
        assert rel(phi, d["phi"]) < 1e-9
        assert rel(ctx2.get_psi(), d["psi"] if variant == "std" else d["psi0"]) < 1e-9
        ctx2.close()


@pytest.mark.parametrize("variant", ["std", "rlm"])
def test_scalar_inflow_layout(variant):
    """alpha_layout 0 (one inflow value for every face and direction) equals the per-face layout holding that
    value, on a rectangular mesh."""
    import copy
    from paper_1907_01027_gb300 import Context, SWEEP_SOURCE
    p = random_problem(20, 4, 0.7, 401, ny=45)
    p.alpha = 0.37
    full = copy.copy(p)
    full.alpha = np.zeros((p.nang, 4, 45, 2))
    full.alpha[..., 0] = 0.37
    x = np.random.default_rng(7).standard_normal((p.nx, 4))
    a, b = Context(p, variant), Context(full, variant)
    ya, yb = a.sweep(x, flags=SWEEP_SOURCE), b.sweep(x, flags=SWEEP_SOURCE)
    assert np.array_equal(ya, yb)
    assert rel(ya, SweepOracle(full).K(variant, x) - _bprime(SweepOracle(full), variant)) < 1e-12
    a.close()
    b.close()


def _bprime(so, variant):
    b = so.rhs(variant)
    if variant == "std":
        return b
    z = so._lm_F()[1] if variant == "lm" else so._rlm_F()[1]
    e = np.zeros((so.nx, 4))
    e[:, 1:] = z
    return b - so.K(variant, e)

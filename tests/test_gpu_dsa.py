"""The vertex diffusion correction on the GPU (lmdg_options.precond = 2 and 3, lmdg_precond_apply) against the
oracle (oracle/vdsa.py): the preconditioner application element by element, and preconditioned solves in the
diffusive regime against the oracle's solutions; with the cell-block step (precond = 3), also in thick cells.

Media: the benchmark's patch medium (sigma_s, sigma_a ~ U[0.1, 10] per patch) on n x n cells of side 1/1024,
i.e. cells of the 1024^2 workload's optical thickness (sigma_t h from 0.1 to 10 at eps = 1e-3)."""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from oracle.vdsa import VertexCorrection
from tests.helpers import rel
from workloads.problems import config4

pytestmark = pytest.mark.gpu


def _medium(n, eps, N=4):
    p = config4(eps=eps, n=n, N=N, patch=max(1, n // 4))
    p.h = 1.0 / 1024
    return p


def _ctx(p, variant, **kw):
    from paper_1907_01027_gb300 import Context
    return Context(p, variant, precond=2, **kw)


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("n,eps", [(16, 1e-3), (37, 1e-2), (64, 1e-3), (70, 1e-3), (1, 1e-3), (2, 1e-2)])
def test_precond_apply_matches_oracle(variant, n, eps):
    """One V-cycle on the device equals the oracle's V-cycle: dense coarsest solves (16, 64: down to 2 x 2 cells;
    1, 2: the fine level is the coarsest) and the damped-Jacobi fallback (37: no coarsening, 38^2 vertices; 70:
    one coarsening to 35, 36^2 vertices times one or two components)."""
    p = _medium(n, eps)
    so = SweepOracle(p)
    b11 = None if variant == "std" else so.B11mat().diagonal().reshape(p.nx, 3)
    ref = VertexCorrection(p, variant, b11, cycles=1)
    ctx = _ctx(p, variant)
    rng = np.random.default_rng(n)
    for _ in range(2):
        x = rng.standard_normal((p.nx, 4))
        assert rel(ctx.precond_apply(x), ref(x).reshape(p.nx, 4)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_preconditioned_solve_matches_direct_16(variant, eps):
    p = _medium(16, eps)
    ref = SweepOracle(p).solve(variant, direct=True)
    ctx = _ctx(p, variant, tol=1e-12, max_iters=5000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0, st
    # two solutions of the same system, the GPU's to a relative residual 1e-12: kappa <= 1e4 here
    assert rel(phi, ref["phi"]) < 1e-8, st
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_preconditioned_solve_matches_oracle_32(variant):
    """32^2 cells, S4, eps = 1e-3: the preconditioned GPU solve against the oracle's (both to 1e-10, the oracle
    with its own vertex correction); two solutions stopped at 1e-10 differ by up to kappa 2e-10."""
    p = _medium(32, 1e-3)
    ref = SweepOracle(p).solve(variant, tol=1e-10, direct=False, precond="vdsa", dsa_cycles=1, maxiter=60)
    assert ref["gmres_info"] == 0
    ctx = _ctx(p, variant, tol=1e-10, max_iters=5000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0, st
    assert rel(phi, ref["phi"]) < 1e-6, st
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm"])
def test_preconditioned_solve_64_fewer_iterations(variant):
    """64^2 cells, S8, eps = 1e-3: to 1e-8 the corrected solve takes under a third of the iterations of the
    Jacobi-scaled one (which is capped at 900)."""
    from paper_1907_01027_gb300 import Context
    p = _medium(64, 1e-3, N=8)
    ctx = _ctx(p, variant, tol=1e-8, max_iters=5000)
    _, _, st, rc = ctx.solve()
    ctx.close()
    assert rc == 0, st
    plain = Context(p, variant, tol=1e-8, max_iters=900)
    _, _, st1, rc1 = plain.solve()
    plain.close()
    assert 3 * st["iters"] <= st1["iters"], (st["iters"], st1["iters"], rc1)


@pytest.mark.parametrize("variant", ["std", "lm"])
def test_mixed_precision_diffusive(variant):
    """FP32 sweeps with FP64 residual sweeps and the vertex correction reach the FP64 residual target at
    eps = 1e-3 and the FP64 solution."""
    from paper_1907_01027_gb300 import FP32, RESID_FP64
    p = _medium(64, 1e-3, N=8)
    c64 = _ctx(p, variant, tol=1e-10)
    _, phi64, st64, rc64 = c64.solve()
    c64.close()
    c32 = _ctx(p, variant, tol=1e-10, precision=FP32, resid=RESID_FP64)
    _, phi32, st, rc = c32.solve()
    c32.close()
    assert rc == 0 and rc64 == 0, (st, st64)
    assert st["resid"] <= 1e-10 * st["resid0"], st
    assert rel(phi32, phi64) < 1e-6, (st, st64)


# ---------------------------------------------------------------- precond = 3: the cell-block Jacobi step

@pytest.mark.parametrize("variant,n,eps,kw", [("std", 16, 1e-3, {}), ("lm", 16, 1e-3, {}), ("rlm", 16, 1e-3, {}),
                                              ("std", 37, 1e-2, {}), ("lm", 37, 1e-2, {}),
                                              ("rlm", 12, 1e-3, {"suppress": 1}), ("std", (24, 13), 1e-3, {}),
                                              ("rlm", (13, 24), 1e-2, {})])
def test_block_precond_apply_matches_oracle(variant, n, eps, kw):
    """y = B^-1 x + C(J x) on the device (blocks from the FP64 sweeps without upwind coupling) against the
    oracle's (blocks by probing its reduced operator, one V-cycle); square and rectangular meshes (the lower left
    n_x x n_y corner of a square medium)."""
    from oracle.vdsa import diagonal_blocks
    if isinstance(n, tuple):
        ni, nj = n
        m = max(ni, nj)
        p = _medium(m, eps)
        p.n, p.ny = ni, nj
        corner = lambda a: np.ascontiguousarray(a.reshape(m, m, *a.shape[1:])[:nj, :ni].reshape(ni * nj, *a.shape[1:]))
        p.sigma_s, p.sigma_a, p.q = corner(p.sigma_s), corner(p.sigma_a), corner(p.q)
        n = ni
    else:
        p = _medium(n, eps)
    so = SweepOracle(p, suppress=bool(kw.get("suppress")))
    b11 = None if variant == "std" else so.B11mat().diagonal().reshape(p.nx, 3)
    ref = VertexCorrection(p, variant, b11, cycles=1, blocks=diagonal_blocks(so, variant))
    from paper_1907_01027_gb300 import Context
    ctx = Context(p, variant, precond=3, **kw)
    rng = np.random.default_rng(p.nx + 3)
    for _ in range(2):
        x = rng.standard_normal((p.nx, 4))
        assert rel(ctx.precond_apply(x), ref(x).reshape(p.nx, 4)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("variant,limit", [("std", 25), ("lm", 80)])
def test_block_precond_thick_cells(variant, limit):
    """64^2 cells of the 256^2 S8 workload at eps = 1e-4 (sigma_t h = 39), S4, to 1e-8: the block step's solve
    converges in a few tens of iterations, fewer than the correction alone, and the oracle certifies it."""
    from paper_1907_01027_gb300 import Context
    from workloads.problems import uniform_problem
    p = uniform_problem(64, 4, 1.0, 1.0, 1.0, eps=1e-4)
    p.h = 1.0 / 256
    c3 = Context(p, variant, precond=3, tol=1e-8, max_iters=3000)
    x, _, st, rc = c3.solve()
    c3.close()
    assert rc == 0 and st["iters"] <= limit, st
    c2 = Context(p, variant, precond=2, tol=1e-8, max_iters=3000)
    _, _, st2, rc2 = c2.solve()
    c2.close()
    assert rc2 == 0 and st["iters"] < st2["iters"], (st, st2)
    so = SweepOracle(p)
    e = np.zeros((p.nx, 4))
    if variant == "lm":
        e[:, 1:] = so._lm_F()[1]
    b = so.rhs(variant)
    assert np.linalg.norm(so.K(variant, x + e) - b) <= 1.5e-8 * np.linalg.norm(b)

"""Pins of the diffusion-correction preconditioner (oracle/dsa.py): the finite-volume operator's stencil,
boundary term and definiteness written out by hand on small meshes, and the preconditioned solves reaching the
direct solution of the same reduced systems with fewer iterations for Q1-DG at eps = 1."""
import numpy as np
import pytest

from oracle.dsa import diffusion_matrix
from oracle.sweeps import SweepOracle
from tests.helpers import rel
from workloads.problems import config4, uniform_problem


def test_constant_medium_stencil_and_boundary():
    # sigma_s = 2, sigma_a = 0, eps = 1: D = 1/6 everywhere, no absorption; interior rows are the 5-point
    # Laplacian times D, boundary faces add 2D / (1 + 4D/h) each
    p = uniform_problem(5, 4, 2.0, 0.0, 1.0)
    A = diffusion_matrix(p).toarray()
    D, h = 1.0 / 6.0, p.h
    Tb = 2 * D / (1 + 4 * D / h)
    c = 2 * 5 + 2                       # cell (2, 2): interior
    assert abs(A[c, c] - 4 * D) < 1e-15
    assert sorted(A[c][A[c] != 0])[:4] == pytest.approx([-D] * 4, abs=1e-15)
    assert abs(A[0, 0] - (2 * D + 2 * Tb)) < 1e-15          # corner: two interior and two boundary faces
    assert abs(A[2, 2] - (3 * D + Tb)) < 1e-15              # edge cell
    assert abs(A.sum() - 20 * Tb) < 1e-13                    # only boundary faces leak (20 of them)


def test_harmonic_mean_symmetric_definite():
    p = uniform_problem(6, 4, 1.0, 0.5, 0.7)
    rng = np.random.default_rng(5)
    p.sigma_s = rng.uniform(0.1, 10, p.nx)
    p.sigma_a = rng.uniform(0.0, 2, p.nx)
    A = diffusion_matrix(p).toarray()
    assert np.allclose(A, A.T, atol=0, rtol=0)
    assert np.linalg.eigvalsh(A).min() > 0
    D = 1 / (3 * (p.sigma_s / p.eps + p.eps * p.sigma_a))
    assert abs(A[0, 1] + 2 * D[0] * D[1] / (D[0] + D[1])) < 1e-15


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_preconditioned_solve(variant):
    # the benchmark's patch statistics on 16 x 16 cells (patches of one cell), S4, eps = 1: the right-
    # preconditioned solve reaches the solution of the unpreconditioned one (both to 1e-12: they differ by at
    # most kappa * 2e-12), in fewer iterations for Q1-DG (15 -> 11) and not more for the low-memory schemes,
    # whose iterations go to the slope block
    p = config4(eps=1.0, n=16, patch=1, N=4)
    so = SweepOracle(p)
    base = so.solve(variant, tol=1e-12, direct=False)
    dsa = so.solve(variant, tol=1e-12, direct=False, precond="dsa")
    assert rel(dsa["phi"], base["phi"]) < 1e-8
    if variant == "std":
        assert dsa["iters"] <= 0.8 * base["iters"], (dsa["iters"], base["iters"])
    else:
        assert dsa["iters"] <= base["iters"] + 2, (dsa["iters"], base["iters"])


def test_multigrid_cycle_contracts():
    """Smoothed-aggregation V-cycles on the benchmark's medium at 64 x 64 cells: the error of the diffusion
    solve falls at least 5x per cycle (against the sparse LU solution)."""
    import scipy.sparse.linalg as spla
    from oracle.dsa import SmoothedAggregation
    p = config4(eps=1.0, n=64, patch=1, N=4)
    A = diffusion_matrix(p).tocsr()
    mg = SmoothedAggregation(A, p.n)
    assert len(mg.levels) == 4                                   # 64 -> 32 -> 16 -> 8 -> 4
    b = np.random.default_rng(1).standard_normal(p.nx)
    exact = spla.spsolve(A.tocsc(), b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(4):
        x = x + mg.vcycle(b - A @ x)
        errs.append(np.linalg.norm(x - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.2 and all(e1 < 0.2 * e0 for e0, e1 in zip(errs, errs[1:])), errs


def test_one_cycle_correction_as_good_as_exact():
    p = config4(eps=1.0, n=16, patch=1, N=4)
    so = SweepOracle(p)
    exact = so.solve("std", tol=1e-12, direct=False, precond="dsa")
    one = so.solve("std", tol=1e-12, direct=False, precond="dsa", dsa_cycles=1)
    assert rel(one["phi"], exact["phi"]) < 1e-8
    assert one["iters"] <= exact["iters"] + 1, (one["iters"], exact["iters"])

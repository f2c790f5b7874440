"""Pins of the vertex diffusion correction (oracle/vdsa.py), the preconditioner of the diffusive regime.

* The cell-average operator's interior row is the nine-point finite-difference form printed for eq-difflimPF
  (golden file), and the full-gradient one the textbook Q1 stencil (8/3 centre, -1/3 neighbours).
* Constants leak through the boundary term only: A 1 sums to the half-range weights times the perimeter.
* Symmetric positive definite on a random medium.
* R_h and I_h: the load of a constant is the hat functions' area; the interpolant of a bilinear function is its
  exact Legendre moments.
* The V-cycle contracts the error of both operators at least 5x per cycle on the benchmark's medium at
  eps = 1e-3, and the cell-average operator needs its two-component coarse space (plain bilinear coarsening
  barely contracts there).
* Preconditioned GMRES reaches the direct solution, and in the diffusive regime takes a few tens of iterations
  where the Jacobi-scaled iteration has not converged after 210.
* The cell-block step: the keyed diagonal blocks equal the dense operator's, cell by cell; with the block step
  the preconditioned spectrum of Q1-DG lies in [0.4, 2.1] at sigma_t h = 3.9 and 3906 (the correction alone
  leaves eigenvalues near 1 / (sigma_t h)); in thick cells it cuts the iterations of Q1-DG and LMDG.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import vdsa
from oracle.sweeps import SweepOracle
from tests.helpers import rel
from workloads.problems import config4, uniform_problem

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lmdg_limit_stencil.txt")


def _kv(path):
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def _row(A, n, I, J):
    nv = n + 1
    r = A.getrow(J * nv + I).toarray().reshape(nv, nv)
    return r[J - 1:J + 2, I - 1:I + 2]


def test_cell_average_row_is_printed_stencil():
    """Interior row of the cell-average operator over h^2 = (diag_coef sum_diag + centre_coef psi) /
    (denominator_factor sigma h^2) + eps sigma_a A[psi], the printed form (with sigma = sigma_t)."""
    g = _kv(GOLD)
    n, ss, sa, eps = 8, 2.0, 0.5, 1.0
    p = uniform_problem(n, 4, ss, sa, 1.0, eps=eps)
    A = vdsa.vertex_matrix(p, "avg")
    h = p.h
    st = _row(A, n, 4, 4) / (h * h)
    sigt = ss / eps + eps * sa
    dc, cc = g["diag_coef"], g["centre_coef"]
    lap = np.array([[dc, 0, dc], [0, cc, 0], [dc, 0, dc]]) / (g["denominator_factor"] * sigt * h * h)
    mass = np.array([[g["A_diag"], g["A_edge"], g["A_diag"]], [g["A_edge"], g["A_centre"], g["A_edge"]],
                     [g["A_diag"], g["A_edge"], g["A_diag"]]])
    assert np.abs(st - (lap + eps * sa * mass)).max() <= 1e-12 * np.abs(st).max()


def test_full_gradient_row_is_q1_stencil():
    n, ss, sa, eps = 8, 1.5, 0.2, 0.5
    p = uniform_problem(n, 4, ss, sa, 1.0, eps=eps)
    A = vdsa.vertex_matrix(p, "full")
    D = 1.0 / (3 * (ss / eps + eps * sa))
    q1 = np.full((3, 3), -1.0 / 3.0)
    q1[1, 1] = 8.0 / 3.0
    mass = np.array([[1, 4, 1], [4, 16, 4], [1, 4, 1]]) / 36.0
    ref = D * q1 + eps * sa * p.h * p.h * mass
    assert np.abs(_row(A, n, 3, 5) - ref).max() <= 1e-15 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["full", "avg"])
def test_constants_leak_through_boundary_only(kind):
    p = uniform_problem(6, 8, 1.0, 0.0, 1.0)
    rng = np.random.default_rng(3)
    p.sigma_s = rng.uniform(0.5, 4.0, p.nx)
    A = vdsa.vertex_matrix(p, kind)
    Ax, Ay = vdsa.half_range_weights(p)
    L = p.n * p.h
    assert abs((A @ np.ones(A.shape[0])).sum() - 2 * (Ax + Ay) * L) <= 1e-13
    assert abs(Ax - Ay) < 1e-14 and 0.2 < Ax < 0.3        # the half-range current of the normalised sphere ~ 1/4


@pytest.mark.parametrize("kind", ["full", "avg"])
def test_symmetric_positive_definite(kind):
    p = uniform_problem(7, 4, 1.0, 0.5, 1.0, eps=0.01)
    rng = np.random.default_rng(4)
    p.sigma_s = rng.uniform(0.1, 10, p.nx)
    p.sigma_a = rng.uniform(0.0, 2, p.nx)
    A = vdsa.vertex_matrix(p, kind).toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_load_and_interpolation():
    p = uniform_problem(5, 4, 1.0, 1.0, 1.0)
    n, h = p.n, p.h
    r = np.zeros((p.nx, 4))
    r[:, 0] = 1.0
    f = vdsa.load(p, r).reshape(n + 1, n + 1)              # sigma_s/eps = 1: int phi_v = area of its cells / 4
    assert np.allclose(f[1:-1, 1:-1], h * h) and np.isclose(f[0, 0], h * h / 4) and np.isclose(f[0, 2], h * h / 2)
    a, b, c, e = 0.3, -1.2, 0.7, 2.5
    xv = p.x0 + np.arange(n + 1) * h
    X, Y = np.meshgrid(xv, xv)
    d = a + b * X + c * Y + e * X * Y
    m = vdsa.interpolate(p, d.ravel()).reshape(n, n, 4)
    xc = p.x0 + (np.arange(n) + 0.5) * h
    Xc, Yc = np.meshgrid(xc, xc)
    # Legendre moments of a + b x + c y + e x y on each cell (xi = 2 (x - xc)/h)
    assert np.allclose(m[:, :, 0], a + b * Xc + c * Yc + e * Xc * Yc, atol=1e-14)
    assert np.allclose(m[:, :, 1], (b + e * Yc) * h / 2, atol=1e-14)
    assert np.allclose(m[:, :, 2], (c + e * Xc) * h / 2, atol=1e-14)
    assert np.allclose(m[:, :, 3], e * h * h / 4, atol=1e-14)


def _medium(n, eps=1e-3, N=4):
    """The benchmark's patch medium on n x n cells of the 1024^2 workload's size h = 1/1024 (so the cells have its
    optical thickness, sigma_t h from 0.1 to 10 at eps = 1e-3)."""
    p = config4(eps=eps, n=n, N=N, patch=max(1, n // 4))
    p.h = 1.0 / 1024
    return p


@pytest.mark.parametrize("kind", ["full", "avg"])
def test_vcycle_contracts(kind):
    p = _medium(64)
    A = vdsa.vertex_matrix(p, kind)
    mg = vdsa.VertexMultigrid(A, p.n, kind)
    assert [lv[3] for lv in mg.levels] == ([1, 1, 1, 1, 1] if kind == "full" else [1, 2, 2, 2, 2])
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    exact = spla.spsolve(A.tocsc(), b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(3):
        x = x + mg.vcycle(b - A @ x)
        errs.append(np.linalg.norm(x - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.2 and all(e1 < 0.2 * e0 for e0, e1 in zip(errs, errs[1:])), errs


def test_cell_average_operator_needs_two_component_coarse_space():
    """With plain bilinear coarsening the checkerboard (-1)^(I+J), nearly in the kernel of the cell-average
    operator, is never corrected: one cycle then leaves most of the error."""
    p = _medium(32)
    A = vdsa.vertex_matrix(p, "avg")
    mg_plain = vdsa.VertexMultigrid(A, p.n, "full")        # same matrix, single-component coarsening
    mg_two = vdsa.VertexMultigrid(A, p.n, "avg")
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    exact = spla.spsolve(A.tocsc(), b)
    e_plain = np.linalg.norm(mg_plain.vcycle(b) - exact) / np.linalg.norm(exact)
    e_two = np.linalg.norm(mg_two.vcycle(b) - exact) / np.linalg.norm(exact)
    assert e_two < 0.2 and e_plain > 0.5, (e_two, e_plain)


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_preconditioned_solve_reaches_direct_solution(variant, eps):
    """8 x 8 cells of the benchmark's optical thickness (sigma_t h from 0.07 to 10): the preconditioned GMRES
    solution to 1e-12 equals the direct (LU) solution within kappa times the tolerance (kappa <= 1e4 here)."""
    p = _medium(8, eps=eps)
    so = SweepOracle(p)
    ref = so.solve(variant, direct=True)
    it = so.solve(variant, tol=1e-12, direct=False, precond="vdsa", dsa_cycles=1, maxiter=300)
    assert it["gmres_info"] == 0 and rel(it["phi"], ref["phi"]) < 1e-8, it["iters"]


@pytest.mark.slow
@pytest.mark.parametrize("variant,limit", [("std", 40), ("lm", 110)])
def test_diffusive_regime_iterations(variant, limit):
    p = _medium(32, N=8)
    so = SweepOracle(p)
    r = so.solve(variant, tol=1e-8, direct=False, precond="vdsa", dsa_cycles=1, maxiter=100)
    assert r["gmres_info"] == 0 and r["iters"] <= limit, r["iters"]
    plain = so.solve(variant, tol=1e-8, direct=False, maxiter=7)      # 7 restart cycles of 30
    assert plain["gmres_info"] != 0


# ---------------------------------------------------------------- cell-block Jacobi step (precond 'bvdsa')

@pytest.mark.parametrize("variant,kw,n,ny", [("std", {}, 6, 5), ("lm", {}, 6, 5), ("rlm", {}, 6, 5),
                                             ("rlm", {"suppress": True}, 8, 0), ("rlm", {"three_cell": True}, 8, 0),
                                             ("rlm", {"q1": True}, 7, 6)])
def test_diagonal_blocks_are_the_operators(variant, kw, n, ny):
    """The keyed probing of diagonal_blocks gives every cell's diagonal block of the dense reduced operator
    (patch media with several materials, rectangles, suppressed faces, the three-cell and Q1-type slopes)."""
    p = config4(eps=1e-2, n=n, N=4, patch=3)
    if ny:   # the first ny rows of the square medium
        p.ny = ny
        p.sigma_s = p.sigma_s[:n * ny].copy()
        p.sigma_a = p.sigma_a[:n * ny].copy()
        p.q = p.q[:n * ny].copy()
    so = SweepOracle(p, **kw)
    K = so.dense_K(variant)
    B = vdsa.diagonal_blocks(so, variant)
    for k in range(p.nx):
        assert np.abs(K[4 * k:4 * k + 4, 4 * k:4 * k + 4] - B[k]).max() <= 1e-14, k


def _thick(n, eps, h):
    p = uniform_problem(n, 4, 1.0, 1.0, 1.0, eps=eps)
    p.h = h
    return p


@pytest.mark.parametrize("sigt_h", [3.9, 3906.0])
def test_block_step_bounds_the_spectrum(sigt_h):
    """Q1-DG, 10 x 10 cells: with the vertex correction alone a fraction of K M's eigenvalues falls to about
    1 / (sigma_t h) -- the modes that change from cell to cell, which no vertex function carries; with the block
    step added every eigenvalue lies in [0.4, 2.1], in thin and in very thick cells alike."""
    eps = 1e-6 if sigt_h > 100 else 1e-3
    p = _thick(10, eps, sigt_h * eps)
    so = SweepOracle(p)
    K = so.dense_K("std")
    n4 = K.shape[0]
    plain = vdsa.VertexCorrection(p, "std")
    block = vdsa.VertexCorrection(p, "std", blocks=vdsa.diagonal_blocks(so, "std"))
    ev_plain = np.linalg.eigvals(K @ np.array([plain(e) for e in np.eye(n4)]).T)
    ev_block = np.linalg.eigvals(K @ np.array([block(e) for e in np.eye(n4)]).T)
    assert np.abs(ev_block).min() >= 0.4 and np.abs(ev_block).max() <= 2.1
    if sigt_h > 100:
        assert np.abs(ev_plain).min() <= 2.0 / sigt_h


@pytest.mark.parametrize("variant,limit_block", [("std", 20), ("lm", 70)])
def test_block_step_in_thick_cells(variant, limit_block):
    """32 x 32 cells with sigma_t h = 39 (the 256^2 S8 workload's cells at eps = 1e-4), to 1e-8: the block step
    cuts the iterations of the corrected solve (Q1-DG 33 -> 14, LMDG 262 -> 54), and both solutions agree."""
    p = _thick(32, 1e-4, 1.0 / 256)
    so = SweepOracle(p)
    a = so.solve(variant, tol=1e-8, direct=False, precond="vdsa", maxiter=20)
    b = so.solve(variant, tol=1e-8, direct=False, precond="bvdsa", maxiter=20)
    assert a["gmres_info"] == 0 and b["gmres_info"] == 0
    assert b["iters"] <= limit_block and b["iters"] < a["iters"], (a["iters"], b["iters"])
    assert rel(a["phi"], b["phi"]) < 1e-4

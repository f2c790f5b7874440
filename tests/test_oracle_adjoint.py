"""Pins of the oracle's adjoint (standard scheme; the paper has no adjoint, the sensitivities are those of the
discrete system eq-sndg-mat with J = sum_K g_K int_K psi_bar).

* The literal transposed sweeps (reverse order, transposed blocks) give the same J and gradients as the dense
  A^T solve on the Appendix A matrices.
* Per direction, L_Omega^T = L_{-Omega} (the transpose of the upwind DG block is the upwind block of the
  opposite direction), which the CUDA adjoint relies on.
* Central finite differences of J agree with the dense adjoint; J is linear in q, so dJ/dq is exact.
"""
import copy

import numpy as np

from oracle import dense
from oracle.sweeps import SweepOracle, adjoint_std
from tests.helpers import random_problem


def _J(p, g):
    L, S, Q = dense.assemble(p)
    psi = np.linalg.solve(L - S, Q).reshape(p.nang, p.nx, 4)
    phi = np.einsum("l,lkr->kr", p.w, psi)
    return float(np.sum(g * p.h * p.h * phi[:, 0]))


def test_sweep_adjoint_equals_dense_adjoint():
    p = random_problem(3, 4, 0.7, 3, q_per_angle=False)
    g = np.random.default_rng(1).uniform(0, 1, p.nx)
    Jd, a, b, c = dense.adjoint_std(p, g)
    Js, a2, b2, c2, _, _ = adjoint_std(SweepOracle(p), g, direct=True)
    assert abs(Jd - Js) <= 1e-13 * abs(Jd)
    for x, y in ((a, a2), (b, b2), (c, c2)):
        assert np.abs(x - y).max() <= 1e-12 * np.abs(x).max()


def test_transpose_is_opposite_direction():
    p = random_problem(4, 8, 0.4, 4)
    so = SweepOracle(p)
    for l in range(p.nang):
        m = np.nonzero((np.abs(p.ox + p.ox[l]) < 1e-15) & (np.abs(p.oy + p.oy[l]) < 1e-15))[0][0]
        u = np.random.default_rng(l).standard_normal((p.nx, 4))
        assert np.abs(so.LT(l, u) / p.w[l] - so.L(m, u) / p.w[m]).max() < 1e-14


def test_dense_adjoint_finite_differences():
    p = random_problem(3, 4, 1.0, 5, q_per_angle=False)
    g = np.random.default_rng(2).uniform(0, 1, p.nx)
    J, dss, dsa, dq = dense.adjoint_std(p, g)
    for K in (0, 4, 7):
        for field, ref in (("sigma_s", dss), ("sigma_a", dsa)):
            d = 1e-4 * getattr(p, field)[K]
            pp, pm = copy.deepcopy(p), copy.deepcopy(p)
            getattr(pp, field)[K] += d
            getattr(pm, field)[K] -= d
            fd = (_J(pp, g) - _J(pm, g)) / (2 * d)
            assert abs(fd - ref[K]) <= 1e-6 * abs(ref[K]), (field, K, fd, ref[K])
        pq = copy.deepcopy(p)
        pq.q[K, 0] += 1.0
        assert abs((_J(pq, g) - J) - dq[K]) <= 1e-12 * max(abs(dq[K]), abs(J))


def test_lowmem_dense_adjoint_finite_differences():
    p = random_problem(3, 4, 1.0, 6, q_per_angle=False)
    g = np.random.default_rng(3).uniform(0, 1, p.nx)
    J, dss, dsa, dq = dense.adjoint(p, g, "lm")
    for K in (0, 5):
        for field, ref in (("sigma_s", dss), ("sigma_a", dsa)):
            d = 1e-4 * getattr(p, field)[K]
            pp, pm = copy.deepcopy(p), copy.deepcopy(p)
            getattr(pp, field)[K] += d
            getattr(pm, field)[K] -= d
            fd = (_Jlm(pp, g) - _Jlm(pm, g)) / (2 * d)
            assert abs(fd - ref[K]) <= 1e-6 * abs(ref[K]), (field, K, fd, ref[K])


def _Jlm(p, g):
    phi = dense.solve(p, "lm")["phi"]
    return float(np.sum(g * p.h * p.h * phi[:, 0]))


def test_reversal_symmetry_holds_for_lm_but_not_rlm():
    """Why the adjoint of RLMDG cannot be solved by the forward sweeps.  With Pi the direction reversal, the full
    form satisfies B^T = Pi B Pi, and V_h^lm is closed under Pi, so the LMDG system A = E^T B E satisfies
    A^T = Pi' A Pi': its adjoint is the forward scheme with the directions reversed (what lmdg_adjoint solves).
    RLMDG is Petrov-Galerkin, A = E^T B Et with the upwind-reconstructed trial basis Et; reversing the directions
    turns upwind into downwind reconstruction, so A^T is a different scheme (O(1) apart)."""
    p = random_problem(3, 4, 0.7, 95, q_per_angle=False)
    L, S, Q = dense.assemble(p)
    B = L - S
    na, nx = p.nang, p.nx
    rev = [int(np.nonzero((np.abs(p.ox + p.ox[l]) < 1e-15) & (np.abs(p.oy + p.oy[l]) < 1e-15))[0][0])
           for l in range(na)]
    full = np.arange(na * nx * 4).reshape(na, nx, 4)
    Pi = np.zeros((na * nx * 4,) * 2)
    Pi[full.ravel(), full[rev].ravel()] = 1.0
    assert np.abs(B.T - Pi @ B @ Pi).max() <= 1e-14 * np.abs(B).max()
    red = np.arange(na * nx).reshape(na, nx)
    perm = np.concatenate([red[rev].ravel(), na * nx + np.arange(3 * nx)])
    E = dense.lm_basis(p)
    A = E.T @ B @ E
    assert np.abs(A.T - A[np.ix_(perm, perm)]).max() <= 1e-13 * np.abs(A).max()
    Et = dense.rlm_trial_basis(p)
    At = E.T @ B @ Et
    assert np.abs(At.T - At[np.ix_(perm, perm)]).max() >= 1e-2 * np.abs(At).max()

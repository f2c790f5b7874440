"""Diffusion-limit and accuracy pins of the oracle (no GPU).

* LMDG as eps -> 0 converges to the nine-point finite-difference system printed in Section 3.1 for
  eq-difflimPF (uniform mesh, constant cross sections), at rate O(eps).
* Q1-DG as eps -> 0 converges to the classical Q1 continuous Galerkin solution of eq-lmdg-cg (Theorem
  thm-sndg-asympscheme), the textbook nine-point Q1 stencil.
* Example examp-2ddifflim: all three schemes keep the limit profile cos(pi x/2) cos(pi y/2) at small eps.
* Table tab-2d-aniso: observed orders of the L1 error of the scalar flux for the fabricated solutions.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.sweeps import SweepOracle
from workloads.problems import Problem, diffusion_limit_problem, mms_sin, mms_aniso
from workloads.quadrature import level_symmetric_2d

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_kv(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = float(line[1])
    return out


def _nodal_problem(n, N, eps, qnode):
    """[-1, 1]^2, sigma_s = sigma_a = 1, zero inflow, q the continuous Q1 interpolant of nodal values."""
    ox, oy, w = level_symmetric_2d(N)
    h = 2.0 / n
    q = np.zeros((n, n, 4))
    f = qnode                                                   # [n+1][n+1] (j, i)
    c00, c10, c01, c11 = f[:-1, :-1], f[:-1, 1:], f[1:, :-1], f[1:, 1:]
    q[..., 0] = (c00 + c10 + c01 + c11) / 4
    q[..., 1] = (c10 + c11 - c00 - c01) / 4
    q[..., 2] = (c01 + c11 - c00 - c10) / 4
    q[..., 3] = (c11 - c10 - c01 + c00) / 4
    nx = n * n
    return Problem(n=n, h=h, x0=-1.0, y0=-1.0, ox=ox, oy=oy, w=w, sigma_s=np.ones(nx), sigma_a=np.ones(nx),
                   q=q.reshape(nx, 4), eps=eps)


def _nodes_from_dg(phi, n):
    """Average of the adjacent cells' Q1 corner values at each node: [n+1][n+1]."""
    P = phi.reshape(n, n, 4)
    acc = np.zeros((n + 1, n + 1))
    cnt = np.zeros((n + 1, n + 1))
    for sj, dj in ((-1, 0), (1, 1)):
        for si, di in ((-1, 0), (1, 1)):
            v = P[..., 0] + si * P[..., 1] + sj * P[..., 2] + si * sj * P[..., 3]
            acc[dj:dj + n, di:di + n] += v
            cnt[dj:dj + n, di:di + n] += 1
    return acc / cnt


def _stencil_solve(n, h, qnode, stiff):
    """Interior-node system stiff(psi) + sigma_a A[psi] = A[q] with homogeneous Dirichlet data."""
    m = n - 1
    idx = lambda i, j: (j - 1) * m + (i - 1)
    A = sp.lil_matrix((m * m, m * m))
    b = np.zeros(m * m)
    g = _read_kv("lmdg_limit_stencil.txt")
    wts = {(0, 0): g["A_centre"]}
    for d in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        wts[d] = g["A_edge"]
    for d in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
        wts[d] = g["A_diag"]
    for j in range(1, n):
        for i in range(1, n):
            r = idx(i, j)
            for (di, dj), c in stiff.items():
                ii, jj = i + di, j + dj
                if 1 <= ii < n and 1 <= jj < n:
                    A[r, idx(ii, jj)] += c
            for (di, dj), c in wts.items():
                ii, jj = i + di, j + dj
                if 1 <= ii < n and 1 <= jj < n:
                    A[r, idx(ii, jj)] += c          # sigma_a = 1
                b[r] += c * qnode[jj, ii]
    sol = spla.spsolve(A.tocsr(), b)
    out = np.zeros((n + 1, n + 1))
    out[1:n, 1:n] = sol.reshape(m, m)
    return out


def _qnode(n):
    x = np.linspace(-1, 1, n + 1)
    X, Y = np.meshgrid(x, x)
    return (np.pi ** 2 / 6 + 1) * np.cos(np.pi * X / 2) * np.cos(np.pi * Y / 2) + 0.3 * X


def test_lmdg_limit_is_printed_stencil():
    n, N = 6, 4
    h = 2.0 / n
    g = _read_kv("lmdg_limit_stencil.txt")
    # -(sum of diagonal neighbours - 4 centre) / (3 sigma_s 2 h^2), sigma_s = 1
    den = 3.0 * g["denominator_factor"] / 3.0 * h * h
    stiff = {(0, 0): g["centre_coef"] / den}
    for d in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
        stiff[d] = g["diag_coef"] / den
    qn = _qnode(n)
    ref = _stencil_solve(n, h, qn, stiff)
    diffs = []
    for eps in (2.0 ** -10, 2.0 ** -14):
        so = SweepOracle(_nodal_problem(n, N, eps, qn))
        phi = so.solve("lm", direct=True)["phi"]
        diffs.append(np.abs(_nodes_from_dg(phi, n) - ref).max() / np.abs(ref).max())
    assert diffs[1] < 2e-4
    assert 8 < diffs[0] / diffs[1] < 32          # O(eps): a 16x smaller eps gives a ~16x smaller gap


def test_q1dg_limit_is_q1_cg():
    n, N = 6, 4
    h = 2.0 / n
    # Q1 continuous Galerkin stiffness int grad phi_i . grad phi_j on squares: centre 8/3, neighbours -1/3,
    # times 1/(3 sigma_s), divided by h^2 like the mass terms.
    stiff = {(0, 0): (8.0 / 3.0) / (3.0 * h * h)}
    for d in ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)):
        stiff[d] = (-1.0 / 3.0) / (3.0 * h * h)
    qn = _qnode(n)
    ref = _stencil_solve(n, h, qn, stiff)
    diffs = []
    for eps in (2.0 ** -10, 2.0 ** -14):
        so = SweepOracle(_nodal_problem(n, N, eps, qn))
        phi = so.solve("std", direct=True)["phi"]
        diffs.append(np.abs(_nodes_from_dg(phi, n) - ref).max() / np.abs(ref).max())
    assert diffs[1] < 2e-4
    assert 8 < diffs[0] / diffs[1] < 32


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_example_diffusion_limit_profile(variant):
    # Example examp-2ddifflim at eps = 2^-10: the cell averages approach cos(pi x/2) cos(pi y/2)
    p = diffusion_limit_problem(10, 4, 2.0 ** -10)
    phi = SweepOracle(p).solve(variant, direct=True)["phi"][:, 0]
    lim = p.info["limit_avg"]
    assert np.abs(phi - lim).max() < 0.06 * lim.max()


def _l1_scalar_flux_error(p, phi, psi_fn):
    g, gw = np.polynomial.legendre.leggauss(5)
    n, h = p.n, p.h
    xc = p.x0 + (np.arange(n) + 0.5) * h
    yc = p.y0 + (np.arange(n) + 0.5) * h
    P = phi.reshape(n, n, 4)
    tot = 0.0
    for a, wa in zip(g, gw):
        for b, wb in zip(g, gw):
            X = xc[None, :] + 0.5 * h * a
            Y = yc[:, None] + 0.5 * h * b
            num = P[..., 0] + P[..., 1] * a + P[..., 2] * b + P[..., 3] * a * b
            ex = sum(p.w[m] * psi_fn(X, Y, p.ox[m], p.oy[m]) for m in range(p.nang))
            tot += np.abs(num - ex).sum() * wa * wb * h * h / 4
    return tot


def _printed_orders():
    out = {}
    for line in open(os.path.join(GOLD, "tab_2d_aniso_orders.txt")):
        t = line.split("#")[0].split()
        if len(t) == 3:
            out[(t[0], t[1])] = float(t[2])
    return out


@pytest.mark.slow
@pytest.mark.parametrize("case", ["sin", "aniso"])
@pytest.mark.parametrize("variant,label", [("std", "Q1-DG"), ("lm", "LMDG"), ("rlm", "RLMDG")])
def test_convergence_orders_table(case, variant, label):
    printed = _printed_orders()[(case, label)]
    errs = []
    for n in (10, 20, 40):
        if case == "sin":
            p = mms_sin(n, 4)
            fn = lambda x, y, a, b: np.sin(x + y)
        else:
            p = mms_aniso(n, 4, c=2.0)
            fn = lambda x, y, a, b: (a - 2.0 * b) ** 2 * np.sin(2 * x + y)
        phi = SweepOracle(p).solve(variant, tol=1e-12, direct=False)["phi"]
        errs.append(_l1_scalar_flux_error(p, phi, fn))
    order = np.log2(errs[1] / errs[2])
    assert abs(order - printed) < 0.15, (errs, order, printed)

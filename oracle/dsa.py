"""Diffusion correction of the cell averages: a right preconditioner for GMRES on the reduced systems.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper leaves preconditioners to future work (its
concluding section); this is the standard diffusion-synthetic construction written out for the schemes here.

The slowly converging modes of the source iteration behind K are smooth and nearly isotropic.  On them the
transport sweep acts like the diffusion operator, L^-1 (sigma_s/eps) phi ~ (D_t)^-1 (sigma_s/eps) phi with
D_t = -div D grad + sigma_t, D = 1 / (3 sigma_t), so I - K ~ (D_t)^-1 D_a with D_a = -div D grad + eps sigma_a
and (I - K)^-1 ~ I + D_a^-1 (sigma_s / eps) on the cell averages.  The correction acts on the average (entry 0
of a cell's reduced unknowns) only.

Discretisation of D_a: cell-centred finite volumes on the uniform mesh, multiplied by the cell area h^2,
    sum_faces T_f (d_K - d_N) + T_b d_K + eps sigma_a,K h^2 d_K = (sigma_s,K / eps) h^2 r_K,
with T_f = 2 D_K D_N / (D_K + D_N) across an interior face (harmonic mean; face length over centre distance
is 1) and T_b = 2 D_K / (1 + 4 D_K / h) on a boundary face: the vacuum condition phi/2 + D dphi/dn = 0 with the
face value eliminated through the one-sided difference over h/2.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def diffusion_matrix(p):
    """The finite-volume matrix of D_a h^2 (sparse, symmetric positive definite) for problem p."""
    n, h, eps = p.n, p.h, p.eps
    ss = np.asarray(p.sigma_s, dtype=float).reshape(n, n)
    sa = np.asarray(p.sigma_a, dtype=float).reshape(n, n)
    D = 1.0 / (3.0 * (ss / eps + eps * sa))
    idx = np.arange(n * n).reshape(n, n)
    rows, cols, vals = [], [], []
    diag = eps * sa * h * h
    for dj, di in ((0, 1), (1, 0)):        # faces between (j, i) and (j + dj, i + di)
        a, b = D[:n - dj, :n - di], D[dj:, di:]
        T = (2.0 * a * b / (a + b)).ravel()
        I, J = idx[:n - dj, :n - di].ravel(), idx[dj:, di:].ravel()
        rows += [I, J, I, J]
        cols += [I, J, J, I]
        vals += [T, T, -T, -T]
    Tb = 2.0 * D / (1.0 + 4.0 * D / h)
    nb = np.zeros((n, n))                  # boundary faces per cell
    nb[0, :] += 1; nb[-1, :] += 1; nb[:, 0] += 1; nb[:, -1] += 1
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append((diag + nb * Tb).ravel())
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n * n, n * n))


class SmoothedAggregation:
    """One V-cycle of smoothed-aggregation multigrid for the finite-volume matrix: the approximate D_a^-1 of
    a device implementation, written out step by step (Vanek, Mandel and Brezina 1996, on the structured mesh).

    Levels: 2 x 2 cell aggregates (n even) give the tentative prolongation P0 (piecewise constant); the
    prolongation P = (I - omega_p D^-1 A) P0 is P0 smoothed by one damped-Jacobi step with omega_p = 2/3; the
    coarse matrix is the Galerkin product P^T A P.  Down to n <= 4 (or an odd n), where a sparse LU solves.  The
    cycle: nu damped-Jacobi steps (omega = 0.8) on the zero guess, the coarse correction of the residual, nu more
    steps."""

    def __init__(self, A, n, nu=2, omega=0.8, omega_p=2.0 / 3.0):
        self.levels = []
        A = sp.csr_matrix(A)
        while n > 4 and n % 2 == 0:
            m = n // 2
            J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            P0 = sp.csr_matrix((np.ones(n * n), ((J * n + I).ravel(), ((J // 2) * m + I // 2).ravel())),
                               shape=(n * n, m * m))
            dinv = 1.0 / A.diagonal()
            P = (P0 - omega_p * (sp.diags(dinv) @ (A @ P0))).tocsr()
            self.levels.append((A, P, dinv))
            A, n = (P.T @ A @ P).tocsr(), m
        self.coarse = spla.splu(A.tocsc())
        self.nu, self.omega = nu, omega

    def vcycle(self, b, level=0):
        if level == len(self.levels):
            return self.coarse.solve(b)
        A, P, dinv = self.levels[level]
        x = np.zeros_like(b)
        for _ in range(self.nu):
            x = x + self.omega * dinv * (b - A @ x)
        x = x + P @ self.vcycle(P.T @ (b - A @ x), level + 1)
        for _ in range(self.nu):
            x = x + self.omega * dinv * (b - A @ x)
        return x


class DiffusionCorrection:
    """v -> v with v[:, 0] += D_a^-1 (sigma_s / eps) v[:, 0]: a sparse LU of the finite-volume matrix
    (``cycles=None``) or that many smoothed-aggregation V-cycles from zero."""

    def __init__(self, p, cycles=None):
        A = diffusion_matrix(p)
        self.cycles = cycles
        if cycles is None:
            self.lu = spla.splu(A)
        else:
            self.A = A.tocsr()
            self.mg = SmoothedAggregation(A, p.n)
        self.src = np.asarray(p.sigma_s, dtype=float) / p.eps * p.h * p.h
        self.nx = p.nx

    def solve(self, r):
        if self.cycles is None:
            return self.lu.solve(r)
        d = np.zeros_like(r)
        for _ in range(self.cycles):
            d = d + self.mg.vcycle(r - self.A @ d)
        return d

    def __call__(self, v):
        w = np.array(v, dtype=float).reshape(self.nx, 4)
        w[:, 0] += self.solve(self.src * w[:, 0])
        return w.ravel()

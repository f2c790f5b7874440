"""Slab-geometry (1D) oracle: the schemes of the paper's one-dimensional tests, assembled and solved directly.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It shares no code with the 2D oracle: the 1D
variational problems are written out here from Section 4.1 (eq-1d) and the definitions of Sections 2-3
restricted to one space dimension.

eq-1d:  mu psi_x + sigma_t psi = (sigma_s / eps) phi + eps q,   sigma_t = sigma_s / eps + eps sigma_a,
        phi = (1/2) int_{-1}^{1} psi dmu,  psi(x_a, mu) = psi_l(mu) for mu > 0,  psi(x_b, mu) = psi_r(mu) for mu < 0.

Discrete ordinates: the N-point Gauss-Legendre rule on [-1, 1] (Section 4.1 uses N = 32), weights halved so
that they sum to one (phi = sum_l w_l psi_l).  Cells K_i of width h, Legendre basis b0 = 1, b1 = xi =
2 (x - x_i) / h.  The upwind DG form of angle l on the full space P1 (Section 2.1 in one dimension):

  a_l(psi, v) = sum_i [ -mu int_K psi v' + mu psi^(x_{i+1/2}) v(x_{i+1/2}^-) - mu psi^(x_{i-1/2}) v(x_{i-1/2}^+)
                        + sigma_t int_K psi v ] - (sigma_s / eps) int phi v,

psi^ the upwind trace (psi_l / psi_r on the inflow boundary, moved to the right-hand side), and the scheme's
global form B(psi, v) = sum_l w_l a_l(psi_l, v_l), Q(v) = sum_l w_l (eps int q_l v_l + inflow terms).

Schemes, each "find psi in the trial space with B(psi, v) = Q(v) for all v in the test space":
  P0-DG   trial = test = piecewise constants per angle;
  P1-DG   trial = test = P1 per angle (the S_N-DG scheme of Section 2.1);
  LMDG    trial = test = V_h^lm: per-angle constants plus one isotropic slope per cell (Section 3.2);
  RLMDG   trial = V_h^lm + R*_alpha (Section 3.3): the per-angle slope reconstructed from the upwind neighbour,
          (h/2) delta = (u_i - u_up) / 2 inside, u_i - psi_inflow on the inflow boundary (the difference over
          h/2), with its angular average removed (R* = R - angular average of R); test = V_h^lm;
  RLMDG*  as RLMDG with the three-cell slope (3 u_i - 4 u_up + u_upup) / 4 from the third cell on (Section 4.1,
          discussion of Example examp-1dfab).
Each system is assembled as S^T A T y = S^T (F - A t0), with A, F the P1 form and functional over all angles,
T (and its affine part t0) the trial basis and S the test basis written as P1 coefficient vectors, and solved
with a sparse direct solver.

Error norm of Tables tab-1d-aniso and tab-1d-eps10-5 (Section 4.1 says only "L1 norm"): the L1 norm of the
angular flux over the slab and the sphere with the normalised angular measure,
sum_l w_l int |psi_h,l(x) - psi(x, mu_l)| dx (40-point Gauss-Legendre rules per cell).  With it the diffusion
table is reproduced to its three printed digits; the scalar-flux L1 norm is not (it is up to 3x smaller).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SCHEMES = ("p0", "p1", "lm", "rlm", "rlm3")


def gauss_ordinates(N):
    """(mu, w): the N-point Gauss-Legendre rule on [-1, 1] with weights summing to 1."""
    mu, w = np.polynomial.legendre.leggauss(N)
    return mu, w / 2.0


class Slab:
    """One slab problem: cross sections (scalars or per-cell arrays), eps, source q(x, mu) (vectorised in x for
    one mu), inflow psi_l(mu) at x_a (mu > 0) and psi_r(mu) at x_b (mu < 0)."""

    def __init__(self, xa, xb, n, N, sigma_s, sigma_a, eps, q, psi_l, psi_r):
        self.xa, self.xb, self.n = float(xa), float(xb), int(n)
        self.h = (self.xb - self.xa) / self.n
        self.xc = self.xa + self.h * (np.arange(self.n) + 0.5)
        self.mu, self.w = gauss_ordinates(N)
        self.nO = N
        self.eps = float(eps)
        self.ss = np.broadcast_to(np.asarray(sigma_s, dtype=float), (self.n,)).copy()
        self.sa = np.broadcast_to(np.asarray(sigma_a, dtype=float), (self.n,)).copy()
        self.st = self.ss / self.eps + self.eps * self.sa
        self.q, self.psi_l, self.psi_r = q, psi_l, psi_r

    # ------------------------------------------------------------------ the P1 form over all angles
    def idx(self, i, l, k):
        """Unknown (cell i, angle l, Legendre coefficient k) of the full P1 space, cell-major."""
        return (i * self.nO + l) * 2 + k

    def full_system(self):
        """A, F with B(psi, v) = v^T A psi and Q(v) = v^T F in P1 coefficients (rows = test functions)."""
        n, nO, h = self.n, self.nO, self.h
        rows, cols, vals = [], [], []
        F = np.zeros(2 * n * nO)
        I = np.arange(n)

        def add(r, c, v):
            r, c = np.broadcast_arrays(np.asarray(r), np.asarray(c))
            rows.append(r.ravel())
            cols.append(c.ravel())
            vals.append(np.broadcast_to(np.asarray(v, dtype=float), r.shape).ravel())

        xg, wg = np.polynomial.legendre.leggauss(8)
        x = self.xc[:, None] + 0.5 * h * xg[None, :]
        for l in range(nO):
            mu, wl = self.mu[l], self.w[l]
            r0, r1 = self.idx(I, l, 0), self.idx(I, l, 1)
            # volume term -mu int psi v': only v = b1 (b1' = 2 / h) against psi's mean: -2 mu c0
            add(r1, r0, -2.0 * mu * wl)
            # collision sigma_t int psi v, int b0 b0 = h, int b1 b1 = h / 3
            add(r0, r0, wl * self.st * h)
            add(r1, r1, wl * self.st * h / 3.0)
            # faces; a cell's trace at its right end is c0 + c1, at its left end c0 - c1
            if mu > 0:
                for r in (r0, r1):            # outflow at the right face, own trace, v(right) = (1, 1)
                    add(r, r0, wl * mu)
                    add(r, r1, wl * mu)
                # inflow at the left face: -mu psi^ v(left), v(left) = (1, -1), psi^ = right trace of cell i - 1
                J = I[1:]
                for r, sgn in ((r0[1:], 1.0), (r1[1:], -1.0)):
                    add(r, self.idx(J - 1, l, 0), -wl * mu * sgn)
                    add(r, self.idx(J - 1, l, 1), -wl * mu * sgn)
                g = self.psi_l(mu)
                F[r0[0]] += wl * mu * g
                F[r1[0]] -= wl * mu * g
            else:
                for r, sgn in ((r0, 1.0), (r1, -1.0)):   # outflow at the left face: -mu (c0 - c1) v(left)
                    add(r, r0, -wl * mu * sgn)
                    add(r, r1, wl * mu * sgn)
                # inflow at the right face: mu psi^ v(right), psi^ = left trace of cell i + 1
                J = I[:-1]
                for r in (r0[:-1], r1[:-1]):
                    add(r, self.idx(J + 1, l, 0), wl * mu)
                    add(r, self.idx(J + 1, l, 1), -wl * mu)
                g = self.psi_r(mu)
                F[r0[-1]] -= wl * mu * g
                F[r1[-1]] -= wl * mu * g
            # source eps int q_l b_m over each cell (8-point Gauss)
            qv = self.q(x, mu)
            F[r0] += wl * self.eps * 0.5 * h * (qv @ wg)
            F[r1] += wl * self.eps * 0.5 * h * (qv @ (wg * xg))
        # scattering -(sigma_s / eps) int phi v, phi = sum_l' w_l' psi_l'
        L, LP = np.meshgrid(np.arange(nO), np.arange(nO), indexing="ij")
        for k, m in ((0, h), (1, h / 3.0)):
            R = self.idx(I[:, None, None], L[None], k)
            C = self.idx(I[:, None, None], LP[None], k)
            V = -(self.ss / self.eps * m)[:, None, None] * (self.w[:, None] * self.w[None, :])[None]
            add(R, C, V)
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(2 * n * nO, 2 * n * nO))
        return A, F

    # ------------------------------------------------------------------ trial / test bases
    def basis(self, scheme):
        """(T, t0, S): trial basis and its affine part, test basis, as P1 coefficient vectors."""
        n, nO = self.n, self.nO
        M = 2 * n * nO
        if scheme == "p1":
            I = sp.identity(M, format="csr")
            return I, np.zeros(M), I
        if scheme == "p0":
            rows = [self.idx(i, l, 0) for i in range(n) for l in range(nO)]
            T = sp.csr_matrix((np.ones(len(rows)), (rows, np.arange(len(rows)))), shape=(M, len(rows)))
            return T, np.zeros(M), T
        # V_h^lm: unknowns per cell [psi0_l for l < nO, X1]
        m = n * (nO + 1)
        rows, cols = [], []
        for i in range(n):
            for l in range(nO):
                rows.append(self.idx(i, l, 0)); cols.append(i * (nO + 1) + l)
                rows.append(self.idx(i, l, 1)); cols.append(i * (nO + 1) + nO)
        Tlm = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(M, m))
        if scheme == "lm":
            return Tlm, np.zeros(M), Tlm
        # reconstruction: slope coefficient (h/2) delta of every (cell, angle) as a combination of the cells'
        # means (and the inflow value on the boundary), then its angular average removed
        three = scheme == "rlm3"
        coef = {}          # (i, l) -> list of (cell, weight) and constant
        const = np.zeros((n, nO))
        for l in range(nO):
            up = -1 if self.mu[l] > 0 else 1          # the upwind neighbour's offset
            gin = self.psi_l(self.mu[l]) if self.mu[l] > 0 else self.psi_r(self.mu[l])
            sgn = 1.0 if self.mu[l] > 0 else -1.0     # delta is d/dx: upwind differences change sign for mu < 0
            for i in range(n):
                first = (i == 0) if up == -1 else (i == n - 1)
                second = (i == 1) if up == -1 else (i == n - 2)
                if first:
                    # (u_i - psi_inflow) over h/2, times h/2
                    terms = [(i, 1.0)]
                    const[i, l] = -sgn * gin
                elif three and not second:
                    terms = [(i, 0.75), (i + up, -1.0), (i + 2 * up, 0.25)]
                else:
                    terms = [(i, 0.5), (i + up, -0.5)]
                coef[(i, l)] = [(c, sgn * wt) for c, wt in terms]
        rows, cols, vals = [], [], []
        t0 = np.zeros(M)
        for i in range(n):
            avg_const = np.sum(self.w * const[i])
            for l in range(nO):
                r = self.idx(i, l, 1)
                t0[r] = const[i, l] - avg_const
                for c, wt in coef[(i, l)]:
                    rows.append(r); cols.append(c * (nO + 1) + l); vals.append(wt)
                for lp in range(nO):
                    for c, wt in coef[(i, lp)]:
                        rows.append(r); cols.append(c * (nO + 1) + lp); vals.append(-self.w[lp] * wt)
        TR = sp.csr_matrix((vals, (rows, cols)), shape=(M, m))
        return (Tlm + TR).tocsr(), t0, Tlm

    def solve(self, scheme):
        """The scheme's solution as per-angle P1 coefficients of the trial function (reconstruction included),
        [n][n_Omega][2]."""
        A, F = self.full_system()
        T, t0, S = self.basis(scheme)
        K = (S.T @ A @ T).tocsc()
        y = spla.spsolve(K, S.T @ (F - A @ t0))
        return (T @ y + t0).reshape(self.n, self.nO, 2)

    def scalar_flux(self, c):
        """phi_h = sum_l w_l psi_h,l as per-cell Legendre coefficients, [n][2]."""
        return np.einsum("l,ilk->ik", self.w, c)

    def l1_error(self, c, psi):
        """sum_l w_l int |psi_h,l - psi(x, mu_l)| dx for a callable psi(x, mu) (40-point Gauss per cell)."""
        xg, wg = np.polynomial.legendre.leggauss(40)
        x = self.xc[:, None] + 0.5 * self.h * xg[None, :]
        e = 0.0
        for l in range(self.nO):
            ph = c[:, l, 0:1] + c[:, l, 1:2] * xg[None, :]
            e += self.w[l] * np.sum(0.5 * self.h * wg[None, :] * np.abs(ph - psi(x, self.mu[l])))
        return float(e)

    def l1_diff(self, c, ref, cref):
        """The same norm of psi_h - psi_ref for a solution cref on a finer slab ref whose cells nest in these."""
        xg, wg = np.polynomial.legendre.leggauss(8)
        x = ref.xc[:, None] + 0.5 * ref.h * xg[None, :]
        i = np.clip(((x - self.xa) / self.h).astype(int), 0, self.n - 1)
        xi = 2.0 * (x - self.xc[i]) / self.h
        e = 0.0
        for l in range(self.nO):
            a = c[i, l, 0] + c[i, l, 1] * xi
            r = cref[:, l, 0:1] + cref[:, l, 1:2] * xg[None, :]
            e += self.w[l] * np.sum(0.5 * ref.h * wg[None, :] * np.abs(a - r))
        return float(e)


# ---------------------------------------------------------------------- the paper's 1D problems
def fabricated(n, case, N=32):
    """Example examp-1dfab: eps = sigma_s = sigma_a = 1 on [0, 1], psi = cos x (case "iso") or cos(x + mu)
    ("aniso"); q and the inflow data follow from psi.  Returns (slab, exact psi(x, mu))."""
    if case == "iso":
        psi = lambda x, mu: np.cos(x) + 0.0 * mu
        dpsi = lambda x, mu: -np.sin(x) + 0.0 * mu
        phi = lambda x: np.cos(x)
    else:
        psi = lambda x, mu: np.cos(x + mu)
        dpsi = lambda x, mu: -np.sin(x + mu)
        phi = lambda x: np.cos(x) * np.sin(1.0)      # (1/2) int_{-1}^{1} cos(x + mu) dmu
    # eps q = mu psi_x + sigma_t psi - (sigma_s / eps) phi with eps = 1, sigma_t = 2
    q = lambda x, mu: mu * dpsi(x, mu) + 2.0 * psi(x, mu) - phi(x)
    s = Slab(0.0, 1.0, n, N, 1.0, 1.0, 1.0, q, lambda mu: psi(0.0, mu), lambda mu: psi(1.0, mu))
    return s, psi


def diffusion_limit(n, eps, N=32):
    """Example examp-1ddifflim: sigma_s = sigma_a = 1 on [0, pi], vacuum inflow, q = (4/3) sin x."""
    q = lambda x, mu: (4.0 / 3.0) * np.sin(x) + 0.0 * mu
    zero = lambda mu: 0.0
    return Slab(0.0, np.pi, n, N, 1.0, 1.0, eps, q, zero, zero)

"""Vertex diffusion correction: a right preconditioner for GMRES on the reduced systems in the diffusive regime.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper leaves preconditioners to future work (its
concluding section); this is the diffusion-synthetic construction written with each scheme's own diffusion limit.

On the slowly converging modes of the source iteration behind K, the transport sweep acts like the diffusion
operator: P L^-1 (sigma_s/eps) ~ D_t^-1 (sigma_s/eps) with D_t = -div D grad + sigma_t, D = 1 / (3 sigma_t),
so K ~ D_t^-1 D_a with D_a = -div D grad + eps sigma_a, and K^-1 ~ I + D_a^-1 (sigma_s / eps).  In the thick
diffusive regime every mode up to the mesh scale is slow, so D_a must be discretised the way each scheme
behaves in its diffusion limit (Section 3.1):

* Q1-DG: the limit is continuous Q1 Galerkin (eq-lmdg-cg, Theorem thm-sndg-asympscheme): stiffness
  int D grad d . grad v on the bilinear vertex functions;
* LMDG, RLMDG: the limit of V_h^lm is eq-difflimPF, the same space with the cell-averaged gradient:
  stiffness int D Pi_0(grad d) . Pi_0(grad v), the nine-point stencil printed for it (only the diagonal
  neighbours of a vertex in the gradient part).

Both add the consistent Q1 mass int eps sigma_a d v and the vacuum (Marshak-type) boundary term
int_{boundary} A_n d v, with A_n = sum_{Omega . n > 0} w Omega . n the half-range outflow weight of the side.

The correction maps a reduced residual r (per cell, Legendre moments) to r + I_h D_a^-1 R_h (sigma_s/eps) r:
R_h tests the cell function (sigma_s/eps) r against the vertex hat functions, I_h takes the vertex solution's
Legendre moments per cell (the bilinear interpolant).  For the low-memory schemes the reduced vector holds
(X0, X1) with the scalar-flux slopes Phi_1 = z - X1, so the correction acts on (r0, -r1) and returns (c0, -c1);
the right preconditioner diag(I, diag(B11))^-1 is applied first.

D_a^-1 is a direct sparse solve, or ``cycles`` V-cycles of the geometric multigrid below (the reference the
device V-cycle is checked against).

In optically thick cells the correction alone loses its effect: the cells are nearly decoupled and scatter
nearly everything back, so modes that change from cell to cell converge as slowly as the smooth ones (K's
eigenvalues there fall to about 1 / (sigma_t h)) and no continuous vertex function carries them.  The block
variant replaces the Jacobi term by the inverse of K's own diagonal blocks (one 4 x 4 block per cell, found by
probing K), which is K to leading order on those modes: v -> B^-1 v + C(J v).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# element matrices on the bilinear corner functions of a square cell, corners ordered (0,0), (1,0), (0,1), (1,1)
_K_FULL = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
_K_AVG = np.array([[2, 0, 0, -2], [0, 2, -2, 0], [0, -2, 2, 0], [-2, 0, 0, 2]]) / 4.0
_M = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) / 36.0
_B = np.array([[2, 1], [1, 2]]) / 6.0


def stiffness_kind(variant):
    """'full' gradient for the standard scheme, cell-average gradient for the low-memory ones."""
    return "full" if variant == "std" else "avg"


def half_range_weights(p):
    """(A_x, A_y): sum of w Omega_x over Omega_x > 0 and of w Omega_y over Omega_y > 0."""
    return float(np.sum(p.w * np.maximum(p.ox, 0.0))), float(np.sum(p.w * np.maximum(p.oy, 0.0)))


def vertex_matrix(p, kind):
    """The vertex matrix of D_a (sparse, symmetric positive definite) on the (n+1) x (m+1) vertices of n x m
    cells, vertex (I, J) at index J (n+1) + I."""
    n, m, h, eps = p.n, p.rows, p.h, p.eps
    ss = np.asarray(p.sigma_s, dtype=float).reshape(m, n)
    sa = np.asarray(p.sigma_a, dtype=float).reshape(m, n)
    D = 1.0 / (3.0 * (ss / eps + eps * sa))
    Ke = _K_FULL if kind == "full" else _K_AVG
    nv = n + 1
    J, I = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    corners = [J * nv + I, J * nv + I + 1, (J + 1) * nv + I, (J + 1) * nv + I + 1]
    rows, cols, vals = [], [], []
    for a in range(4):
        for b in range(4):
            rows.append(corners[a].ravel())
            cols.append(corners[b].ravel())
            vals.append((D * Ke[a, b] + eps * sa * h * h * _M[a, b]).ravel())
    Ax, Ay = half_range_weights(p)
    k, kj = np.arange(n), np.arange(m)
    for e0, e1, c in ((k, k + 1, Ay), (m * nv + k, m * nv + k + 1, Ay),          # south, north sides
                      (kj * nv, (kj + 1) * nv, Ax), (kj * nv + n, (kj + 1) * nv + n, Ax)):   # west, east sides
        for a, ea in enumerate((e0, e1)):
            for b, eb in enumerate((e0, e1)):
                rows.append(ea)
                cols.append(eb)
                vals.append(np.full(len(ea), c * h * _B[a, b]))
    nvv = nv * (m + 1)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nvv, nvv))


def load(p, r):
    """f_v = int (sigma_s/eps) r phi_v over the cells touching vertex v, r given as Legendre moments [n_x][4]."""
    n, m, h = p.n, p.rows, p.h
    s = (np.asarray(p.sigma_s, dtype=float) / p.eps).reshape(m, n)
    R = np.asarray(r, dtype=float).reshape(m, n, 4) * s[:, :, None]
    f = np.zeros((m + 1, n + 1))
    for cy, dj in ((-1, 0), (1, 1)):
        for cx, di in ((-1, 0), (1, 1)):
            # int_K b_m phi_c = h^2/4 (1, cx/3, cy/3, cx cy/9) for the corner c = (cx, cy) of the reference square
            f[dj:dj + m, di:di + n] += h * h / 4.0 * (R[:, :, 0] + R[:, :, 1] * cx / 3.0 + R[:, :, 2] * cy / 3.0
                                                       + R[:, :, 3] * cx * cy / 9.0)
    return f.ravel()


def interpolate(p, d):
    """Legendre moments [n_x][4] of the bilinear interpolant of the vertex values d."""
    n, m = p.n, p.rows
    d = np.asarray(d, dtype=float).reshape(m + 1, n + 1)
    d00, d10, d01, d11 = d[:m, :n], d[:m, 1:], d[1:, :n], d[1:, 1:]
    out = np.zeros((m, n, 4))
    out[:, :, 0] = (d00 + d10 + d01 + d11) / 4.0
    out[:, :, 1] = (-d00 + d10 - d01 + d11) / 4.0
    out[:, :, 2] = (-d00 - d10 + d01 + d11) / 4.0
    out[:, :, 3] = (d00 - d10 - d01 + d11) / 4.0
    return out.reshape(n * m, 4)


def _interp_1d(nc):
    """Linear interpolation from nc + 1 coarse to 2 nc + 1 fine points (dense rows)."""
    P = np.zeros((2 * nc + 1, nc + 1))
    for i in range(2 * nc + 1):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, i // 2] = P[i, i // 2 + 1] = 0.5
    return sp.csr_matrix(P)


class VertexMultigrid:
    """Geometric multigrid V-cycle for the vertex matrix, written out step by step.

    Levels halve the cells along x and y while both numbers are even and above 2.  Prolongation: bilinear
    interpolation of every component.  For the cell-average stiffness, whose gradient part couples only
    diagonal neighbours (the vertices with I + J even and odd are two decoupled lattices, joined only by the mass
    and boundary terms, so the checkerboard (-1)^(I+J) is nearly in its kernel), the first coarsening carries two
    components per coarse vertex: P = [P_bl, C P_bl] with C = diag((-1)^(I+J)), i.e. functions smooth on each of
    the two lattices; coarser levels interpolate both components bilinearly.  Coarse matrices are Galerkin
    products P^T A P.  Smoothing: ``nu`` damped block-Jacobi steps (``omega``) before and after the coarse
    correction, starting from zero; the coarsest level is solved exactly (dense inverse, at most ``max_dense``
    unknowns; larger coarsest levels take ``coarse_sweeps`` damped-Jacobi steps instead)."""

    def __init__(self, A, n, kind, m=None, nu=2, omega=0.7, max_dense=1156, coarse_sweeps=50):
        self.nu, self.omega, self.coarse_sweeps = nu, omega, coarse_sweeps
        self.levels = []                   # (A, P to the next coarser level, block-diagonal inverse, bs)
        A = sp.csr_matrix(A)
        m = n if m is None else m
        bs = 1
        while n % 2 == 0 and m % 2 == 0 and n > 2 and m > 2:
            nc, mc = n // 2, m // 2
            Pbl = sp.kron(_interp_1d(mc), _interp_1d(nc)).tocsr()   # index J (n+1) + I, both levels
            if bs == 1 and kind == "avg":
                J, I = np.divmod(np.arange((n + 1) * (m + 1)), n + 1)
                C = sp.diags(np.where((I + J) % 2 == 0, 1.0, -1.0))
                P = sp.hstack([Pbl, C @ Pbl]).tocsr()               # coarse unknowns [all a ; all b]
                P = P @ _interleave(Pbl.shape[1], 2)                 # reorder to [vertex][component]
                bsc = 2
            else:
                P = sp.kron(Pbl, sp.identity(bs)).tocsr()
                bsc = bs
            self.levels.append((A, P, _block_diag_inv(A, bs), bs))
            A = (P.T @ A @ P).tocsr()
            n, m, bs = nc, mc, bsc
        self.coarse_A, self.coarse_bs = A, bs
        if A.shape[0] <= max_dense:
            self.coarse_inv = np.linalg.inv(A.toarray())
        else:
            self.coarse_inv = None
            self.coarse_dinv = _block_diag_inv(A, bs)

    def _smooth(self, A, dinv, bs, b, x, steps):
        for _ in range(steps):
            r = b - A @ x
            x = x + self.omega * _block_apply(dinv, r, bs)
        return x

    def vcycle(self, b, level=0):
        if level == len(self.levels):
            if self.coarse_inv is not None:
                return self.coarse_inv @ b
            return self._smooth(self.coarse_A, self.coarse_dinv, self.coarse_bs, b, np.zeros_like(b),
                                self.coarse_sweeps)
        A, P, dinv, bs = self.levels[level]
        x = self._smooth(A, dinv, bs, b, np.zeros_like(b), self.nu)
        x = x + P @ self.vcycle(P.T @ (b - A @ x), level + 1)
        return self._smooth(A, dinv, bs, b, x, self.nu)


def _interleave(nv, bs):
    """Permutation matrix taking [component][vertex] order to [vertex][component]."""
    idx = np.arange(nv * bs)
    comp, vert = np.divmod(idx, nv)
    return sp.csr_matrix((np.ones(nv * bs), (idx, vert * bs + comp)), shape=(nv * bs, nv * bs))


def _block_diag_inv(A, bs):
    A = sp.csr_matrix(A)
    nv = A.shape[0] // bs
    out = np.zeros((nv, bs, bs))
    for c in range(bs):
        for d in range(bs):
            out[:, c, d] = A[np.arange(nv) * bs + c, np.arange(nv) * bs + d].A1
    return np.linalg.inv(out)


def _block_apply(dinv, r, bs):
    return np.einsum("vcd,vd->vc", dinv, r.reshape(-1, bs)).ravel()


def block_key(so, variant, k):
    """What the diagonal block of cell k depends on: the cell's own solve sees its material (sigma_s, sigma_a),
    and with the upwind reconstruction of RLMDG also which of its faces lie on the boundary -- the distance to each
    side, up to 2 for the three-cell slopes of RLMDG* -- and which faces are suppressed."""
    p = so.p
    key = (float(p.sigma_s[k]), float(p.sigma_a[k]))
    if variant == "rlm":
        i, j = k % p.n, k // p.n
        key += (min(i, 2), min(p.n - 1 - i, 2), min(j, 2), min(p.rows - 1 - j, 2))
        if so.supp is not None:
            key += (int(so.supp[k]),)
    return key


def diagonal_blocks(so, variant):
    """The diagonal blocks of the reduced operator K of ``variant`` (the homogeneous map of ``so.K``): [n_x][4][4],
    column r of cell k's block the cell-k part of K e_(k, r).  K applied to a vector that lives in one cell reaches
    that cell only through its own solve (every other cell it reaches lies downwind), so the block is the same for
    cells with the same ``block_key``; one cell per key is probed with four applications of K."""
    nx = so.p.nx
    B = np.zeros((nx, 4, 4))
    seen = {}
    for k in range(nx):
        key = block_key(so, variant, k)
        if key not in seen:
            blk = np.zeros((4, 4))
            for r in range(4):
                e = np.zeros((nx, 4))
                e[k, r] = 1.0
                blk[:, r] = so.K(variant, e)[k]
            seen[key] = blk
        B[k] = seen[key]
    return B


class VertexCorrection:
    """The right preconditioner v -> J v + C(J v) on reduced vectors [n_x][4] for a variant, with J the Jacobi
    scaling diag(I, diag(B11))^-1 of the low-memory schemes (``b11diag``: [n_x][3], None for the standard
    scheme) and C the vertex diffusion correction, its solve direct (``cycles=None``) or by that many V-cycles
    from zero.

    With ``blocks`` (the diagonal blocks of K, :func:`diagonal_blocks`) the first term is the cell-block Jacobi
    step instead: v -> B^-1 v + C(J v).  In optically thick cells most of K's slow modes vary from cell to cell
    (the cells are nearly decoupled and scatter nearly everything back), which no continuous vertex function
    represents; on these the block of K is K to leading order, and B^-1 takes them to eigenvalues near 1 while
    C takes the smooth ones."""

    def __init__(self, p, variant, b11diag=None, cycles=None, blocks=None, **mg):
        self.p, self.variant, self.cycles = p, variant, cycles
        self.kind = stiffness_kind(variant)
        self.A = vertex_matrix(p, self.kind)
        self.b11diag = b11diag
        self.binv = None if blocks is None else np.linalg.inv(blocks)
        if cycles is None:
            self.lu = spla.splu(self.A.tocsc())
        else:
            self.mg = VertexMultigrid(self.A, p.n, self.kind, m=p.rows, **mg)

    def solve(self, f):
        if self.cycles is None:
            return self.lu.solve(f)
        d = np.zeros_like(f)
        for _ in range(self.cycles):
            d = d + self.mg.vcycle(f - self.A @ d)
        return d

    def correction(self, u):
        """I_h D_a^-1 R_h (sigma_s/eps) u for a cell function u [n_x][4] (scalar-flux moments)."""
        return interpolate(self.p, self.solve(load(self.p, u)))

    def __call__(self, v):
        v = np.array(v, dtype=float).reshape(self.p.nx, 4)
        u = v.copy()
        if self.variant != "std":
            u[:, 1:] /= self.b11diag
            phi = u.copy()
            phi[:, 1:] *= -1.0
            c = self.correction(phi)
            c[:, 1:] *= -1.0
        else:
            c = self.correction(u)
        first = u if self.binv is None else np.einsum("krs,ks->kr", self.binv, v)
        return (first + c).ravel()

"""Problem instances: meshes, media, sources and inflow data for eq-main on 2D Cartesian meshes.

Everything here is input data.  The scaled equation (eq-main) is

    Omega . grad Psi + (sigma_s / eps + eps sigma_a) Psi = (sigma_s / eps) Psi_bar + eps q,   Psi = alpha on Gamma^-,

and the manufactured-solution helpers below evaluate its *continuous* residual to build ``q`` (Section 4.2
fabricated solutions); the discretisation is not involved.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .quadrature import level_symmetric_2d

_D = np.array([1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0])   # int b_r^2 over the reference square / 4


@dataclass
class Problem:
    n: int                       # cells along x
    h: float
    x0: float
    y0: float
    ox: np.ndarray
    oy: np.ndarray
    w: np.ndarray
    sigma_s: np.ndarray          # [n_x]
    sigma_a: np.ndarray          # [n_x]
    q: np.ndarray                # [n_x][4] (layout 1) or [n_Omega][n_x][4] (layout 2)
    eps: float = 1.0
    alpha: Optional[np.ndarray] = None   # [n_Omega][4][max(n, rows)][2] or None for vacuum (see face_count)
    name: str = ""
    info: dict = field(default_factory=dict)
    ny: int = 0                  # cells along y (0: n, a square mesh)

    @property
    def rows(self):
        """Cells along y."""
        return self.ny or self.n

    @property
    def nx(self):
        """Number of cells."""
        return self.n * self.rows

    def face_count(self, side):
        """Boundary faces of a side (0 west, 1 east: one per row; 2 south, 3 north: one per column).  ``alpha``
        holds a side's faces in its first face_count(side) entries."""
        return self.rows if side < 2 else self.n

    @property
    def nang(self):
        return len(self.w)

    @property
    def q_layout(self):
        return 2 if self.q.ndim == 3 else 1

    def cell_centres(self):
        c = self.x0 + (np.arange(self.n) + 0.5) * self.h
        d = self.y0 + (np.arange(self.rows) + 0.5) * self.h
        X, Y = np.meshgrid(c, d)          # [j][i]
        return X.ravel(), Y.ravel()


def _gauss(npts):
    return np.polynomial.legendre.leggauss(npts)


def legendre_project_cell(f, n, h, x0, y0, npts=5):
    """Q1 Legendre coefficients of ``f(x, y)`` on every cell: returns ``[n*n][4]`` (cell index j*n + i)."""
    g, gw = _gauss(npts)
    xc = x0 + (np.arange(n) + 0.5) * h
    yc = y0 + (np.arange(n) + 0.5) * h
    out = np.zeros((n, n, 4))
    for a, (ga, wa) in enumerate(zip(g, gw)):
        for b, (gb, wb) in enumerate(zip(g, gw)):
            X = xc[None, :] + 0.5 * h * ga
            Y = yc[:, None] + 0.5 * h * gb
            fv = f(X, Y) * (wa * wb / 4.0)
            out[:, :, 0] += fv
            out[:, :, 1] += fv * ga
            out[:, :, 2] += fv * gb
            out[:, :, 3] += fv * ga * gb
    return (out / _D).reshape(n * n, 4)


def legendre_project_face(f, n, h, x0, y0, npts=5):
    """Linear Legendre coefficients of ``f(x, y)`` on the boundary faces: returns ``[4][n][2]``.

    Sides: 0 west (x = x0), 1 east, 2 south (y = y0), 3 north.  Face coordinate t runs along +y on the
    west/east sides and along +x on the south/north sides.
    """
    g, gw = _gauss(npts)
    c = (np.arange(n) + 0.5) * h
    out = np.zeros((4, n, 2))
    L = n * h
    for t, wt in zip(g, gw):
        s = c + 0.5 * h * t
        vals = [f(np.full(n, x0), y0 + s), f(np.full(n, x0 + L), y0 + s),
                f(x0 + s, np.full(n, y0)), f(x0 + s, np.full(n, y0 + L))]
        for side, v in enumerate(vals):
            out[side, :, 0] += 0.5 * wt * v
            out[side, :, 1] += 1.5 * wt * v * t
    return out


def uniform_problem(n, N, sigma_s, sigma_a, q, eps=1.0, L=1.0, x0=0.0, y0=0.0, name="", ny=0):
    """n x ny cells (ny = 0: n x n) of side L / n, constant media and source, S_N level-symmetric, vacuum."""
    ox, oy, w = level_symmetric_2d(N)
    nx = n * (ny or n)
    qq = np.zeros((nx, 4))
    qq[:, 0] = q
    return Problem(n=n, h=L / n, x0=x0, y0=y0, ox=ox, oy=oy, w=w,
                   sigma_s=np.full(nx, float(sigma_s)), sigma_a=np.full(nx, float(sigma_a)),
                   q=qq, eps=eps, alpha=None, name=name, ny=ny)


def config1():
    """32x32 cells, S4, sigma_s = 1, sigma_a = 0.5, q = 1, eps = 1, vacuum inflow."""
    return uniform_problem(32, 4, 1.0, 0.5, 1.0, name="std-32x32-S4")


def config2(eps=1.0):
    """256x256 cells, S8, sigma_s = sigma_a = 1, q = 1, vacuum inflow; eps in {1, 1e-2, 1e-4}."""
    return uniform_problem(256, 8, 1.0, 1.0, 1.0, eps=eps, name=f"256x256-S8-eps{eps:g}")


def config3():
    """512x512 cells, S12: 7x7 block pattern, absorbing blocks (sigma_s = 0, sigma_a = 10) in a scatterer
    (sigma_s = 1, sigma_a = 0), q = 1 in the centre block only, eps = 1, vacuum inflow.

    Block (a, b) = (floor(7 x), floor(7 y)) of the cell centre; it absorbs iff a + b is even, neither a nor b
    is 0 or 6, and (a, b) != (3, 3)  (an interior checkerboard around the source block).
    """
    n = 512
    p = uniform_problem(n, 12, 1.0, 0.0, 0.0, name="rlm-512x512-S12-blocks")
    X, Y = p.cell_centres()
    a = np.floor(7 * X).astype(int)
    b = np.floor(7 * Y).astype(int)
    absorb = ((a + b) % 2 == 0) & (a > 0) & (a < 6) & (b > 0) & (b < 6) & ~((a == 3) & (b == 3))
    p.sigma_s = np.where(absorb, 0.0, 1.0)
    p.sigma_a = np.where(absorb, 10.0, 0.0)
    p.q[:, 0] = np.where((a == 3) & (b == 3), 1.0, 0.0)
    return p


def config4(eps=1.0, seed=1907, n=1024, N=16, patch=16):
    """1024x1024 cells, S16, sigma_s and sigma_a piecewise constant on 16x16-cell patches, each drawn
    U[0.1, 10] from ``numpy.random.default_rng(seed)`` (all sigma_s patches first, patch-major, then all
    sigma_a patches), q = 1, vacuum inflow; eps in {1, 1e-3}."""
    p = uniform_problem(n, N, 1.0, 1.0, 1.0, eps=eps, name=f"{n}x{n}-S{N}-patch{patch}-eps{eps:g}")
    rng = np.random.default_rng(seed)
    npch = -(-n // patch)                  # patches per side (the last one partial when patch does not divide n)
    ss = rng.uniform(0.1, 10.0, npch * npch).reshape(npch, npch)
    sa = rng.uniform(0.1, 10.0, npch * npch).reshape(npch, npch)
    jj, ii = np.meshgrid(np.arange(n) // patch, np.arange(n) // patch, indexing="ij")
    p.sigma_s = ss[jj, ii].ravel().copy()
    p.sigma_a = sa[jj, ii].ravel().copy()
    return p


def config5(n=256, N=8, seed=1907):
    """256x256 cells, S8, sigma_s = 1 + sum of 8 Gaussian bumps a exp(-|x - c|^2 / w^2) sampled at cell
    centres (c ~ U[0,1]^2, then a ~ U[0, 2], then w ~ U[0.05, 0.2], all from default_rng(seed)),
    sigma_a = 0.1, q = 1, eps = 1, vacuum inflow.  ``info['detector']`` marks cells with centre x > 0.9."""
    p = uniform_problem(n, N, 1.0, 0.1, 1.0, name=f"adjoint-{n}x{n}-S{N}-bumps")
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, (8, 2))
    a = rng.uniform(0.0, 2.0, 8)
    wd = rng.uniform(0.05, 0.2, 8)
    X, Y = p.cell_centres()
    s = np.ones_like(X)
    for k in range(8):
        s += a[k] * np.exp(-((X - c[k, 0]) ** 2 + (Y - c[k, 1]) ** 2) / wd[k] ** 2)
    p.sigma_s = s
    p.info["detector"] = (X > 0.9).astype(np.float64)
    p.info["fd_cells"] = np.sort(np.random.default_rng(seed + 1).choice(p.nx, 32, replace=False))
    return p


def mms_problem(n, N, psi, dpsi_dx, dpsi_dy, sigma_s=1.0, sigma_a=1.0, eps=1.0, L=1.0, x0=0.0, y0=0.0,
                npts=5, name="mms"):
    """Manufactured solution ``psi(x, y, ox, oy)``: builds the angle-dependent source from the continuous
    residual of eq-main (with the discrete angular average, as in eq:sn) and ``alpha = psi`` on the
    boundary.  ``info['phi_avg']`` holds the exact cell averages of the scalar flux.  ``sigma_s`` and
    ``sigma_a`` are numbers or functions of (x, y) constant on every cell (a layered or patched medium)."""
    ox, oy, w = level_symmetric_2d(N)
    h = L / n
    nang = len(w)
    ss = sigma_s if callable(sigma_s) else (lambda x, y, v=float(sigma_s): v + 0 * x)
    sa = sigma_a if callable(sigma_a) else (lambda x, y, v=float(sigma_a): v + 0 * x)

    def psibar(x, y):
        return sum(w[m] * psi(x, y, ox[m], oy[m]) for m in range(nang))

    q = np.zeros((nang, n * n, 4))
    alpha = np.zeros((nang, 4, n, 2))
    for l in range(nang):
        a, b = ox[l], oy[l]

        def ql(x, y, a=a, b=b):
            sig_t = ss(x, y) / eps + eps * sa(x, y)
            return (a * dpsi_dx(x, y, a, b) + b * dpsi_dy(x, y, a, b) + sig_t * psi(x, y, a, b)
                    - (ss(x, y) / eps) * psibar(x, y)) / eps
        q[l] = legendre_project_cell(ql, n, h, x0, y0, npts)
        alpha[l] = legendre_project_face(lambda x, y, a=a, b=b: psi(x, y, a, b), n, h, x0, y0, npts)
    phi = legendre_project_cell(psibar, n, h, x0, y0, npts)[:, 0]
    xc = x0 + (np.arange(n) + 0.5) * h
    yc = y0 + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, yc)                     # [j][i]
    return Problem(n=n, h=h, x0=x0, y0=y0, ox=ox, oy=oy, w=w,
                   sigma_s=np.asarray(ss(X, Y), dtype=float).ravel(),
                   sigma_a=np.asarray(sa(X, Y), dtype=float).ravel(), q=q, eps=eps, alpha=alpha, name=name,
                   info={"phi_avg": phi})


def mms_sin(n, N, **kw):
    """Isotropic fabricated solution psi = sin(x + y) (Section 4.2, first case)."""
    return mms_problem(n, N, lambda x, y, a, b: np.sin(x + y), lambda x, y, a, b: np.cos(x + y),
                       lambda x, y, a, b: np.cos(x + y), name="mms-sin", **kw)


def mms_aniso(n, N, c=3.0, **kw):
    """Anisotropic fabricated solution psi = (Omega_x - c Omega_y)^2 sin(2x + y); the text prints c = 3 and
    the table c = 2 (Section 4.2)."""
    return mms_problem(n, N, lambda x, y, a, b: (a - c * b) ** 2 * np.sin(2 * x + y),
                       lambda x, y, a, b: 2 * (a - c * b) ** 2 * np.cos(2 * x + y),
                       lambda x, y, a, b: (a - c * b) ** 2 * np.cos(2 * x + y), name=f"mms-aniso{c:g}", **kw)


def diffusion_limit_problem(n, N, eps):
    """Section 4.2 diffusion-limit example on [-1, 1]^2: sigma_s = sigma_a = 1, zero inflow,
    q = (pi^2/6 + 1) cos(pi x / 2) cos(pi y / 2); the limit solution is cos(pi x / 2) cos(pi y / 2)."""
    ox, oy, w = level_symmetric_2d(N)
    h = 2.0 / n
    qf = lambda x, y: (np.pi ** 2 / 6 + 1) * np.cos(np.pi * x / 2) * np.cos(np.pi * y / 2)
    q = legendre_project_cell(qf, n, h, -1.0, -1.0)
    lim = legendre_project_cell(lambda x, y: np.cos(np.pi * x / 2) * np.cos(np.pi * y / 2), n, h, -1.0, -1.0)
    nx = n * n
    return Problem(n=n, h=h, x0=-1.0, y0=-1.0, ox=ox, oy=oy, w=w, sigma_s=np.ones(nx), sigma_a=np.ones(nx),
                   q=q, eps=eps, alpha=None, name=f"difflim-eps{eps:g}", info={"limit_avg": lim[:, 0]})

"""Dense brute-force oracle: the S_N-DG variational problems assembled and solved directly.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Tiny meshes only: the full space V_h has
n_Omega * n_x * 4 unknowns and the matrix is dense.

What it computes (paper sections cited per function):

* standard S_N-DG, eq-sndg-scheme: find psi in V_h with B(psi, v) = Q_alpha(v) for all v in V_h;
* low-memory LMDG, eq-gene-scheme: the same with trial = test = V_h^lm = V_{h,0} + D_{h,1} (Section 3.2);
* reconstructed RLMDG, eq-rlmdg-vari: find psi in V_h^lm with B(psi + R*_alpha psi, v) = Q_alpha(v) for all v
  in V_h^lm (Section 3.3); the affine part of R*_alpha is moved to the right-hand side.

Entries follow Appendix A: L carries the factor w_l, S = M P has entries w_l w_l' int sigma_s/eps b b, and
Q carries w_l.  Every integral is evaluated with 3-point Gauss-Legendre rules on the physical cell or face
(exact for the polynomial integrands), from basis functions evaluated pointwise.
"""
import numpy as np

_G, _GW = np.polynomial.legendre.leggauss(3)


def _basis(xi, eta):
    """Legendre Q1 basis (b0, b1, b2, b3) = (1, xi, eta, xi*eta) at reference points."""
    xi = np.asarray(xi, dtype=float)
    eta = np.asarray(eta, dtype=float)
    return np.stack([np.ones_like(xi), xi, eta, xi * eta])


def _basis_grad(xi, eta, h):
    """Physical gradients (d/dx, d/dy) of the basis: d/dx = (2/h) d/dxi."""
    xi = np.asarray(xi, dtype=float)
    eta = np.asarray(eta, dtype=float)
    z = np.zeros_like(xi)
    o = np.ones_like(xi)
    dx = np.stack([z, o, z, eta]) * (2.0 / h)
    dy = np.stack([z, z, o, xi]) * (2.0 / h)
    return dx, dy


def _ref_integrals(h):
    """Cell and face integrals of the basis on a square cell of side h (Appendix A building blocks).

    mass[r][s]  = int_K b_s b_r dx
    vol[d][r][s] = int_K b_s d_d b_r dx            (d = x, y)
    face f in (W, E, S, N) with outward normal nu_f:
      self[f][r][s] = int_F b_s^K b_r^K ds         (both traces from inside K)
      nbr[f][r][s]  = int_F b_s^K' b_r^K ds        (K' = neighbour across F)
    """
    XI, ETA = np.meshgrid(_G, _G, indexing="ij")
    WW = np.outer(_GW, _GW) * (h * h / 4.0)
    B = _basis(XI, ETA)
    dX, dY = _basis_grad(XI, ETA, h)
    mass = np.einsum("rab,sab,ab->rs", B, B, WW)
    vol = np.stack([np.einsum("rab,sab,ab->rs", dX, B, WW), np.einsum("rab,sab,ab->rs", dY, B, WW)])
    fw = _GW * (h / 2.0)
    # (own reference coordinates on the face, neighbour's reference coordinates on the same points)
    faces = {
        0: ((-np.ones(3), _G), (np.ones(3), _G)),     # west: own xi=-1, neighbour's xi=+1
        1: ((np.ones(3), _G), (-np.ones(3), _G)),     # east
        2: ((_G, -np.ones(3)), (_G, np.ones(3))),     # south
        3: ((_G, np.ones(3)), (_G, -np.ones(3))),     # north
    }
    selfF = np.zeros((4, 4, 4))
    nbrF = np.zeros((4, 4, 4))
    for f, (own, nb) in faces.items():
        Bo = _basis(*own)
        Bn = _basis(*nb)
        selfF[f] = np.einsum("ra,sa,a->rs", Bo, Bo, fw)
        nbrF[f] = np.einsum("ra,sa,a->rs", Bo, Bn, fw)
    normals = np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, -1.0], [0.0, 1.0]])
    return mass, vol, selfF, nbrF, normals


def _neighbour(n, m, i, j, f):
    """Neighbour (i', j') across face f of cell (i, j) on n x m cells, or None on the boundary."""
    if f == 0:
        return (i - 1, j) if i > 0 else None
    if f == 1:
        return (i + 1, j) if i < n - 1 else None
    if f == 2:
        return (i, j - 1) if j > 0 else None
    return (i, j + 1) if j < m - 1 else None


def _face_alpha_integrals(alpha_l, n, i, j, f, h):
    """int_F alpha b_r^K ds for the boundary face f of cell (i, j); alpha = a0 + a1 t along the face."""
    if f in (0, 1):
        a0, a1 = alpha_l[f, j]
        t = _G                                            # t follows +y, the cell's eta on this face
        xi = -np.ones(3) if f == 0 else np.ones(3)
        B = _basis(xi, _G)
    else:
        a0, a1 = alpha_l[f, i]
        t = _G
        eta = -np.ones(3) if f == 2 else np.ones(3)
        B = _basis(_G, eta)
    return B @ ((a0 + a1 * t) * _GW) * (h / 2.0)


def assemble(p):
    """Global matrices of Appendix A on the full space V_h: returns (Lmat, Smat, Qvec) with B = L - S.

    Index of the basis function xi^{l,p,r}: (l * n_x + p) * 4 + r, cell p = j * n + i (n cells along x, m along y).
    """
    n, m, h, nx, na = p.n, p.rows, p.h, p.nx, p.nang
    mass, vol, selfF, nbrF, normals = _ref_integrals(h)
    sig_t = p.sigma_s / p.eps + p.eps * p.sigma_a
    dim = na * nx * 4
    L = np.zeros((dim, dim))
    S = np.zeros((dim, dim))
    Q = np.zeros(dim)
    for l in range(na):
        om = np.array([p.ox[l], p.oy[l]])
        wl = p.w[l]
        for j in range(m):
            for i in range(n):
                K = j * n + i
                rows = slice((l * nx + K) * 4, (l * nx + K) * 4 + 4)
                # volume: -int u Omega.grad v + int sigma_t u v   (eq-Ljk)
                L[rows, rows] += wl * (-(om[0] * vol[0] + om[1] * vol[1]) + sig_t[K] * mass)
                for f in range(4):
                    on = om @ normals[f]
                    nb = _neighbour(n, m, i, j, f)
                    if on > 0:                             # outflow: upwind trace is the interior one
                        L[rows, rows] += wl * on * selfF[f]
                    elif nb is not None:                   # inflow from the neighbour
                        Kn = nb[1] * n + nb[0]
                        cols = slice((l * nx + Kn) * 4, (l * nx + Kn) * 4 + 4)
                        L[rows, cols] += wl * on * nbrF[f]
                    elif p.alpha is not None:              # inflow boundary: -int alpha Omega.nu v
                        Q[rows] += -wl * on * _face_alpha_integrals(p.alpha[l], n, i, j, f, h)
                qK = p.q[l, K] if p.q.ndim == 3 else p.q[K]
                Q[rows] += wl * p.eps * (mass @ qK)
    # S = M P: S[(l,p,r),(l',p,s)] = w_l w_l' int sigma_s/eps b_s b_r   (Appendix A)
    for K in range(nx):
        blk = (p.sigma_s[K] / p.eps) * mass
        for l in range(na):
            rows = slice((l * nx + K) * 4, (l * nx + K) * 4 + 4)
            for m in range(na):
                cols = slice((m * nx + K) * 4, (m * nx + K) * 4 + 4)
                S[rows, cols] += p.w[l] * p.w[m] * blk
    return L, S, Q


def _same_material(p):
    """(sx, sy): sx[j, f] is True when cells (f, j) and (f + 1, j) have equal (sigma_s, sigma_a), sy[f, i]
    likewise for cells (i, f) and (i, f + 1)."""
    n, m = p.n, p.rows
    ss, sa = p.sigma_s.reshape(m, n), p.sigma_a.reshape(m, n)
    sx = (ss[:, 1:] == ss[:, :-1]) & (sa[:, 1:] == sa[:, :-1])
    sy = (ss[1:, :] == ss[:-1, :]) & (sa[1:, :] == sa[:-1, :])
    return sx, sy


def reconstruct(p, u0, alpha, suppress=False, three_cell=False, q1=False):
    """Upwind reconstruction R_alpha Pi_0 (Section 3.3.1): 2D P1 slopes, and with ``q1`` the Q1-type term.

    ``u0``: cell averages ``[n_Omega][n_x]``.  Returns the Legendre coefficients ``[n_Omega][n_x][4]`` of
    (delta_x u)(x - x_i) + (delta_y u)(y - y_j): coefficient of b1 = xi is (h/2) delta_x, of b2 = eta is
    (h/2) delta_y.  delta uses the upwind side s_x = -sign(Omega_x); at the inflow boundary the difference is
    taken with alpha at the face midpoint over a spacing h/2 (alpha None means 0).  The face-midpoint value
    of the linear face data (a0 + a1 t) is a0.  ``suppress``: no reconstruction across an interior face where
    the cross sections jump (the remedy Section 4 applies to the kinks at a discontinuity): the upwind
    difference across such a face is zero.  ``three_cell`` (RLMDG*, Section 4.1): from the third cell on,
    delta is the slope at the cell centre of the quadratic with the cell averages of the cell and its two upwind
    neighbours, (3 u_i - 4 u_{i-1} + u_{i-2}) / (2h); the second cell keeps the two-cell difference and the
    inflow cell the boundary difference.  ``q1`` (the Q1-type reconstruction Section 3.3.1 mentions without a
    formula; reading of this oracle): also the coefficient (h/2)^2 delta_xy of b3 = xi eta, delta_xy the upwind
    y-difference of the reconstructed x-slopes delta_x, (delta_x(j) - delta_x(j -+ 1)) / h, and on the y-inflow
    boundary row (delta_x - d alpha/dx) / (h/2) with d alpha/dx = 2 a1 / h along that boundary face (alpha None:
    0); exact for bilinear functions, which the two-cell P1 reconstruction is not.
    """
    n, m, h, na = p.n, p.rows, p.h, p.nang
    out = np.zeros((na, n * m, 4))
    same_x, same_y = _same_material(p) if suppress else (None, None)
    for l in range(na):
        U = u0[l].reshape(m, n)              # [j][i]
        dx = np.zeros((m, n))
        dy = np.zeros((m, n))
        if p.ox[l] > 0:                      # delta^-_x
            dx[:, 1:] = (U[:, 1:] - U[:, :-1]) / h
            if three_cell:
                dx[:, 2:] = (3 * U[:, 2:] - 4 * U[:, 1:-1] + U[:, :-2]) / (2 * h)
            aW = alpha[l, 0, :m, 0] if alpha is not None else np.zeros(m)
            dx[:, 0] = (U[:, 0] - aW) / (h / 2)
        else:                                # delta^+_x
            dx[:, :-1] = (U[:, 1:] - U[:, :-1]) / h
            if three_cell:
                dx[:, :-2] = -(3 * U[:, :-2] - 4 * U[:, 1:-1] + U[:, 2:]) / (2 * h)
            aE = alpha[l, 1, :m, 0] if alpha is not None else np.zeros(m)
            dx[:, -1] = (aE - U[:, -1]) / (h / 2)
        if p.oy[l] > 0:
            dy[1:, :] = (U[1:, :] - U[:-1, :]) / h
            if three_cell:
                dy[2:, :] = (3 * U[2:, :] - 4 * U[1:-1, :] + U[:-2, :]) / (2 * h)
            aS = alpha[l, 2, :n, 0] if alpha is not None else np.zeros(n)
            dy[0, :] = (U[0, :] - aS) / (h / 2)
        else:
            dy[:-1, :] = (U[1:, :] - U[:-1, :]) / h
            if three_cell:
                dy[:-2, :] = -(3 * U[:-2, :] - 4 * U[1:-1, :] + U[2:, :]) / (2 * h)
            aN = alpha[l, 3, :n, 0] if alpha is not None else np.zeros(n)
            dy[-1, :] = (aN - U[-1, :]) / (h / 2)
        if suppress:
            if p.ox[l] > 0:
                dx[:, 1:] *= same_x
            else:
                dx[:, :-1] *= same_x
            if p.oy[l] > 0:
                dy[1:, :] *= same_y
            else:
                dy[:-1, :] *= same_y
        out[l, :, 1] = (h / 2) * dx.ravel()
        out[l, :, 2] = (h / 2) * dy.ravel()
        if q1:
            dxy = np.zeros((m, n))
            if p.oy[l] > 0:
                dxy[1:, :] = (dx[1:, :] - dx[:-1, :]) / h
                gS = 2.0 * alpha[l, 2, :n, 1] / h if alpha is not None else np.zeros(n)
                dxy[0, :] = (dx[0, :] - gS) / (h / 2)
            else:
                dxy[:-1, :] = (dx[1:, :] - dx[:-1, :]) / h
                gN = 2.0 * alpha[l, 3, :n, 1] / h if alpha is not None else np.zeros(n)
                dxy[-1, :] = (gN - dx[-1, :]) / (h / 2)
            out[l, :, 3] = (h / 2) ** 2 * dxy.ravel()
    return out


def _Rstar(p, u0, alpha, suppress=False, three_cell=False, q1=False):
    """R*_alpha applied to the piecewise constants u0: R_alpha Pi_0 u minus its angular average."""
    R = reconstruct(p, u0, alpha, suppress, three_cell, q1)
    return R - np.einsum("l,lkr->kr", p.w, R)[None]


def p0_basis(p):
    """Basis matrix of V_{h,0} (Section 3.1): the per-direction cell constants xi^{l,p,0}."""
    na, nx = p.nang, p.nx
    E = np.zeros((na * nx * 4, na * nx))
    for l in range(na):
        for K in range(nx):
            E[(l * nx + K) * 4, l * nx + K] = 1.0
    return E


def lm_basis(p):
    """Basis matrix of V_h^lm: columns xi^{l,p,0} (l, p) then eta^{p,r} = sum_l xi^{l,p,r} (p, r = 1..3)."""
    na, nx = p.nang, p.nx
    dim = na * nx * 4
    E = np.zeros((dim, na * nx + 3 * nx))
    for l in range(na):
        for K in range(nx):
            E[(l * nx + K) * 4, l * nx + K] = 1.0
    for K in range(nx):
        for r in range(1, 4):
            c = na * nx + K * 3 + (r - 1)
            for l in range(na):
                E[(l * nx + K) * 4 + r, c] = 1.0
    return E


def rlm_trial_basis(p, suppress=False, three_cell=False, q1=False):
    """Trial basis of V_h^rlm: xi^{l,p,0} + R*_0 xi^{l,p,0}, then eta^{p,r} (Section 3.3.2)."""
    na, nx = p.nang, p.nx
    E = lm_basis(p)
    Et = E.copy()
    for l in range(na):
        for K in range(nx):
            u0 = np.zeros((na, nx))
            u0[l, K] = 1.0
            Rs = _Rstar(p, u0, None, suppress, three_cell, q1)
            Et[:, l * nx + K] += Rs.ravel()
    return Et


def solve(p, variant, suppress=False, three_cell=False, q1=False):
    """Solve the discrete problem (``suppress``: RLMDG without reconstruction across cross-section jumps;
    ``three_cell``: RLMDG* with the three-cell reconstruction).
    Returns a dict with

    ``psi``  full coefficients [n_Omega][n_x][4] of the (reconstructed) discrete solution,
    ``phi``  scalar flux moments sum_l w_l psi_l, [n_x][4],
    ``psi0``, ``phi1`` (low-memory variants) the V_h^lm coefficients: per-angle cell averages and the
    isotropic slopes.
    """
    L, S, Q = assemble(p)
    B = L - S
    na, nx = p.nang, p.nx
    out = {}
    if variant == "std":
        psi = np.linalg.solve(B, Q).reshape(na, nx, 4)
    elif variant == "p0":
        E = p0_basis(p)
        c = np.linalg.solve(E.T @ B @ E, E.T @ Q)
        psi = (E @ c).reshape(na, nx, 4)
        out["psi0"] = c.reshape(na, nx)
    elif variant == "lm":
        E = lm_basis(p)
        c = np.linalg.solve(E.T @ B @ E, E.T @ Q)
        psi = (E @ c).reshape(na, nx, 4)
        out["psi0"] = c[:na * nx].reshape(na, nx)
        out["phi1"] = c[na * nx:].reshape(nx, 3)
    elif variant == "rlm":
        E = lm_basis(p)
        Et = rlm_trial_basis(p, suppress, three_cell, q1)
        rho = _Rstar(p, np.zeros((na, nx)), p.alpha, suppress, three_cell, q1).ravel()   # affine part R*_alpha 0
        c = np.linalg.solve(E.T @ B @ Et, E.T @ (Q - B @ rho))
        psi = (Et @ c + rho).reshape(na, nx, 4)
        out["psi0"] = c[:na * nx].reshape(na, nx)
        out["phi1"] = c[na * nx:].reshape(nx, 3)
    else:
        raise ValueError(variant)
    out["psi"] = psi
    out["phi"] = np.einsum("l,lkr->kr", p.w, psi)
    return out


def operator_matrices(p):
    """(L, S, Q) of Appendix A, exposed for adjoint and invariant checks."""
    return assemble(p)


def adjoint_std(p, g):
    """Dense adjoint of the standard scheme: A = L - S and Q of Appendix A; A Psi = Q; J = G^T Psi with
    G_(l,K,r) = w_l g_K int_K b_r; A^T lam = G; dJ/dp = lam^T (dQ/dp - dA/dp Psi).  A and Q are affine in each
    sigma_s, sigma_a and q value, so dA/dp and dQ/dp are differences of two assemblies (exact up to rounding)."""
    import copy
    L, S, Q = assemble(p)
    A = L - S
    psi = np.linalg.solve(A, Q)
    na, nx = p.nang, p.nx
    mass = _ref_integrals(p.h)[0]
    Gv = np.zeros(na * nx * 4)
    for l in range(na):
        for K in range(nx):
            Gv[(l * nx + K) * 4:(l * nx + K) * 4 + 4] = p.w[l] * g[K] * mass[:, 0]
    J = float(Gv @ psi)
    lam = np.linalg.solve(A.T, Gv)
    out = []
    for field in ("sigma_s", "sigma_a", "q"):
        d = np.zeros(nx)
        for K in range(nx):
            p2 = copy.deepcopy(p)
            if field == "q":
                if p2.q.ndim == 3:
                    p2.q[:, K, 0] += 1.0
                else:
                    p2.q[K, 0] += 1.0
            else:
                getattr(p2, field)[K] += 1.0
            L2, S2, Q2 = assemble(p2)
            d[K] = lam @ ((Q2 - Q) - ((L2 - S2) - A) @ psi)
        out.append(d)
    return J, out[0], out[1], out[2]


def adjoint(p, g, variant):
    """Dense adjoint of the standard or low-memory scheme: the discrete system is (E^T B E) c = E^T Q with E the
    trial/test basis (identity for the standard scheme, the V_h^lm basis for LMDG); J = G^T E c with
    G_(l,K,r) = w_l g_K int_K b_r; (E^T B E)^T mu = E^T G; dJ/dp = mu^T E^T (dQ/dp - dB/dp E c), with dB, dQ
    differences of affine assemblies."""
    import copy
    L, S, Q = assemble(p)
    B = L - S
    na, nx = p.nang, p.nx
    E = np.eye(na * nx * 4) if variant == "std" else lm_basis(p)
    mass = _ref_integrals(p.h)[0]
    Gv = np.zeros(na * nx * 4)
    for l in range(na):
        for K in range(nx):
            Gv[(l * nx + K) * 4:(l * nx + K) * 4 + 4] = p.w[l] * g[K] * mass[:, 0]
    A = E.T @ B @ E
    c = np.linalg.solve(A, E.T @ Q)
    psi = E @ c
    J = float(Gv @ psi)
    mu = np.linalg.solve(A.T, E.T @ Gv)
    out = []
    for field in ("sigma_s", "sigma_a", "q"):
        dd = np.zeros(nx)
        for K in range(nx):
            p2 = copy.deepcopy(p)
            if field == "q":
                if p2.q.ndim == 3:
                    p2.q[:, K, 0] += 1.0
                else:
                    p2.q[K, 0] += 1.0
            else:
                getattr(p2, field)[K] += 1.0
            L2, S2, Q2 = assemble(p2)
            dd[K] = mu @ (E.T @ ((Q2 - Q) - ((L2 - S2) - B) @ psi))
        out.append(dd)
    return J, out[0], out[1], out[2]

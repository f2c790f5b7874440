"""Sweep-based FP64 oracle: the paper's reduced systems built from its block operators, step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper.  Per-angle blocks carry the Appendix A weight w_l: (L Psi)_l = w_l Lhat_l psi_l,
(M Phi)_l = w_l int sigma_s/eps b b Phi, Q_l = w_l (int eps q_l b - int_{inflow boundary} alpha Omega.nu b),
P = weighted angular sum, Sigma = unweighted angular sum, Sigma^T = copy to every angle.  Lhat_l and its
inverses come from ``csweep.c``.

* Standard S_N-DG (Section 2.1.1): K Phi = Phi - P L^-1 M Phi, right-hand side P L^-1 Q (eq-sndg-phi),
  recovery Psi = L^-1 (M Phi + Q) (eq-sndg-final-sweep).
* LMDG (Section 3.2): B11 = Sigma L11 Sigma^T - Sigma M1 (eq-lmdg-psi1), K applied as eq-nonrec-block,
  right-hand side of eq-lmdg-reducemat, recovery eq-lm-step4.
* RLMDG (Section 3.3.2), read as follows where the printed system is inconsistent: the tilde blocks and
  Q-tilde as printed;
  with X1 = (B11^-1 Sigma Ltilde10 + P1 R) Psi0 the second block row of the reduced operator and of the
  right-hand side is G' = Sigma Ltilde10 + B11 P1 R (= B11 times the printed row's operator), which is what
  applying Sigma Ltilde10 to eq-rlmdg-psi0 and closing with X1 produces; recovery Psi0 = Ltilde00^-1
  (M0 X0 + L01 Sigma^T X1) + Ltilde00^-1 (Qtilde0 - L01 Sigma^T B11^-1 Sigma Qtilde1) and eq-rlmdg-psi1.

B11^-1 is applied with conjugate gradients (B11 is SPD for centrally symmetric quadratures, Theorem
lem-B11); the reduced systems are solved with scipy's GMRES or, for small meshes, by a dense LU of the
operator built column by column.
"""
import ctypes
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import scipy.sparse.linalg as spla

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("osw_apply_L", "osw_sweep_L", "osw_sweep_L00", "osw_apply_LT", "osw_sweep_LT"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            f.restype = None
        lib.osw_sweep_Lt00.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       dp, dp, dp, ctypes.POINTER(ctypes.c_ubyte), ctypes.c_int]
        lib.osw_sweep_Lt00.restype = None
        lib.osw_elem_tables.argtypes = [ctypes.c_double, dp]
        lib.osw_elem_tables.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def elem_tables(h):
    out = np.zeros(240)
    _load().osw_elem_tables(h, _ptr(out))
    return {"mass": out[:16].reshape(4, 4), "vol": out[16:48].reshape(2, 4, 4),
            "self": out[48:112].reshape(4, 4, 4), "nbr": out[112:176].reshape(4, 4, 4)}


class SweepOracle:
    """Matrix-free block operators of one problem.  ``threads`` angles are processed concurrently; every
    angular sum is accumulated in angle order, so results do not depend on the thread count."""

    def __init__(self, p, threads=None, literal_b11=False, suppress=False, three_cell=False, q1=False):
        """``suppress``: RLMDG without reconstruction across cross-section jumps; ``three_cell``: RLMDG* (the
        three-cell upwind reconstruction from the third cell on); ``q1``: the Q1-type reconstruction (also the
        xi eta coefficient, see ``R``)."""
        self.p = p
        self.literal_b11 = literal_b11
        self.three_cell = three_cell
        self.q1 = q1
        self.n, self.m, self.h, self.nx, self.na = p.n, p.rows, p.h, p.nx, p.nang
        self.suppress = suppress
        self.supp = self._suppression_bits() if suppress else None
        self.sigt = np.ascontiguousarray(p.sigma_s / p.eps + p.eps * p.sigma_a, dtype=np.float64)
        self.sse = p.sigma_s / p.eps
        self.mass = elem_tables(p.h)["mass"]
        self.threads = threads or (os.cpu_count() or 1)
        self.lib = _load()
        self.cg_iters = 0

    def _suppression_bits(self):
        """Interior faces where (sigma_s, sigma_a) jumps: per cell, bit 1 west, 2 east, 4 south, 8 north.  With
        ``suppress`` the RLMDG reconstruction takes no difference across these faces (the remedy for the kinks
        at cross-section discontinuities, Section 4)."""
        n, m, p = self.n, self.m, self.p
        ss, sa = p.sigma_s.reshape(m, n), p.sigma_a.reshape(m, n)
        bits = np.zeros((m, n), dtype=np.uint8)
        for j in range(m):
            for i in range(n):
                for bit, (jj, ii) in ((1, (j, i - 1)), (2, (j, i + 1)), (4, (j - 1, i)), (8, (j + 1, i))):
                    if 0 <= ii < n and 0 <= jj < m and (ss[j, i] != ss[jj, ii] or sa[j, i] != sa[jj, ii]):
                        bits[j, i] |= bit
        return bits.ravel()

    # ---------------------------------------------------------------- per-angle primitives (Lhat_l)
    def _call(self, name, l, a, size):
        out = np.zeros(size)
        a = np.ascontiguousarray(a, dtype=np.float64)
        args = [self.n, self.m, self.h, float(self.p.ox[l]), float(self.p.oy[l]), _ptr(self.sigt), _ptr(a),
                _ptr(out)]
        if name == "osw_sweep_Lt00":
            args.append(None if self.supp is None else self.supp.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
            args.append(1 if self.three_cell else 0)
        getattr(self.lib, name)(*args)
        return out

    def L(self, l, u):
        """(L u)_l = w_l Lhat_l u for a [n_x][4] vector u."""
        return self.p.w[l] * self._call("osw_apply_L", l, u.ravel(), 4 * self.nx).reshape(self.nx, 4)

    def Linv(self, l, b):
        """(L^-1 b)_l: solves w_l Lhat_l u = b by an upwind sweep."""
        return self._call("osw_sweep_L", l, b.ravel() / self.p.w[l], 4 * self.nx).reshape(self.nx, 4)

    def LT(self, l, u):
        """(L^T u)_l = w_l Lhat_l^T u."""
        return self.p.w[l] * self._call("osw_apply_LT", l, u.ravel(), 4 * self.nx).reshape(self.nx, 4)

    def LTinv(self, l, b):
        """Solves w_l Lhat_l^T u = b by the reverse-order transposed sweep."""
        return self._call("osw_sweep_LT", l, b.ravel() / self.p.w[l], 4 * self.nx).reshape(self.nx, 4)

    def L00inv(self, l, b0):
        return self._call("osw_sweep_L00", l, b0 / self.p.w[l], self.nx)

    def Lt00inv(self, l, b0):
        return self._call("osw_sweep_Lt00", l, b0 / self.p.w[l], self.nx)

    def M(self, l, Phi):
        """(M Phi)_l = w_l int sigma_s/eps b_r b_s Phi_s (Appendix A), Phi: [n_x][4]."""
        return self.p.w[l] * self.sse[:, None] * (Phi @ self.mass.T)

    def Q(self, l):
        """Q_l = w_l (int eps q_l b_r - sum over inflow boundary faces of int alpha Omega_l.nu b_r)."""
        p = self.p
        qK = p.q[l] if p.q.ndim == 3 else p.q
        out = p.eps * (qK @ self.mass.T)
        if p.alpha is not None:
            out = out + self._boundary(l)
        return p.w[l] * out

    def _boundary(self, l):
        p, n, m, h = self.p, self.n, self.m, self.h
        g, gw = np.polynomial.legendre.leggauss(3)
        out = np.zeros((m, n, 4))                    # [j][i][r]
        ox, oy = p.ox[l], p.oy[l]
        # (side, Omega.nu, cell slice, own reference coordinates of the face points, faces of the side)
        sides = [(0, -ox, (slice(None), 0), (-np.ones(3), g), m), (1, ox, (slice(None), n - 1), (np.ones(3), g), m),
                 (2, -oy, (0, slice(None)), (g, -np.ones(3)), n), (3, oy, (m - 1, slice(None)), (g, np.ones(3)), n)]
        for side, on, sl, (xi, eta), nf in sides:
            if on >= 0:
                continue
            B = np.stack([np.ones(3), xi, eta, xi * eta])           # [r][pt]
            a = p.alpha[l, side, :nf]                               # [faces][2]
            vals = a[:, 0:1] + a[:, 1:2] * g[None, :]               # [face][pt]
            integ = (vals * gw[None, :]) @ B.T * (h / 2.0)          # [face][r]
            out[sl] += -on * integ
        return out.reshape(self.nx, 4)

    def _angles_sum(self, fn, shape, weights=None):
        """sum_l fn(l) (weights None) accumulated in angle order over concurrent chunks."""
        acc = np.zeros(shape)
        with ThreadPoolExecutor(self.threads) as ex:
            for c0 in range(0, self.na, self.threads):
                res = list(ex.map(fn, range(c0, min(self.na, c0 + self.threads))))
                for r in res:
                    acc += r
        return acc

    def _angles_map(self, fn):
        with ThreadPoolExecutor(self.threads) as ex:
            return list(ex.map(fn, range(self.na)))

    # ---------------------------------------------------------------- standard S_N-DG (Section 2.1.1)
    def K_std(self, Phi):
        Phi = Phi.reshape(self.nx, 4)
        PLM = self._angles_sum(lambda l: self.p.w[l] * self.Linv(l, self.M(l, Phi)), (self.nx, 4))
        return Phi - PLM

    def rhs_std(self):
        return self._angles_sum(lambda l: self.p.w[l] * self.Linv(l, self.Q(l)), (self.nx, 4))

    def recover_std(self, Phi):
        Phi = Phi.reshape(self.nx, 4)
        return np.stack(self._angles_map(lambda l: self.Linv(l, self.M(l, Phi) + self.Q(l))))

    # ---------------------------------------------------------------- low-memory blocks (Section 3.2)
    def _slopes(self, X1):
        u = np.zeros((self.nx, 4))
        u[:, 1:] = X1
        return u

    def _const(self, psi0):
        u = np.zeros((self.nx, 4))
        u[:, 0] = psi0
        return u

    def M0(self, l, X0):
        return self.p.w[l] * self.sse * self.mass[0, 0] * X0

    def L01SigT(self, l, X1):
        return self.L(l, self._slopes(X1))[:, 0]

    def SigL10(self, Psi0):
        return self._angles_sum(lambda l: self.L(l, self._const(Psi0[l]))[:, 1:], (self.nx, 3))

    def P0(self, Psi0):
        return np.einsum("l,lk->k", self.p.w, Psi0)

    def B11(self, X1):
        """B11 X1 = Sigma L11 Sigma^T X1 - Sigma M1 X1 (eq-lmdg-psi1)."""
        X1 = X1.reshape(self.nx, 3)
        SL = self._angles_sum(lambda l: self.L(l, self._slopes(X1))[:, 1:], (self.nx, 3))
        SM = self._angles_sum(lambda l: self.M(l, self._slopes(X1))[:, 1:], (self.nx, 3))
        return SL - SM

    def B11mat(self):
        """B11 assembled once by probing the matrix-free operator above (see ``_b11_sparse``)."""
        if getattr(self, "_B11", None) is None:
            self._B11 = _b11_sparse(self)
            self._B11lu = None
        return self._B11

    def B11fast(self, X1):
        if self.literal_b11:
            return self.B11(X1)
        return (self.B11mat() @ X1.reshape(-1)).reshape(self.nx, 3)

    def B11inv(self, r, rtol=1e-15):
        if self.nx <= 200_000:
            import scipy.sparse.linalg as _sl
            self.B11mat()
            if self._B11lu is None:
                self._B11lu = _sl.splu(self._B11.tocsc())
            return self._B11lu.solve(np.ascontiguousarray(r.reshape(-1))).reshape(self.nx, 3)
        n3 = 3 * self.nx
        op = spla.LinearOperator((n3, n3), matvec=lambda v: self.B11fast(v).ravel(), dtype=np.float64)
        its = [0]
        x, info = spla.cg(op, r.ravel(), rtol=rtol, atol=0.0, maxiter=20 * n3,
                          callback=lambda xk: its.__setitem__(0, its[0] + 1))
        self.cg_iters += its[0]
        return x.reshape(self.nx, 3)

    def SigQ1(self, Qt1=None):
        return self._angles_sum(lambda l: self.Q(l)[:, 1:], (self.nx, 3))

    # ---------------------------------------------------------------- LMDG reduced system
    def K_lm(self, X):
        """eq-nonrec-block: K [X0; X1] = [X0; B11 X1] - [P0; Sigma L10] L00^-1 (M0 X0 + L01 Sigma^T X1)."""
        X = X.reshape(self.nx, 4)
        X0, X1 = X[:, 0], X[:, 1:]
        Psi0 = np.stack(self._angles_map(lambda l: self.L00inv(l, self.M0(l, X0) + self.L01SigT(l, X1))))
        out = np.zeros((self.nx, 4))
        out[:, 0] = X0 - self.P0(Psi0)
        out[:, 1:] = self.B11fast(X1) - self.SigL10(Psi0)
        return out

    def _lm_F(self):
        """L00^-1 (Q0 - L01 Sigma^T B11^-1 Sigma Q1) and z = B11^-1 Sigma Q1."""
        z = self.B11inv(self.SigQ1())
        F = np.stack(self._angles_map(lambda l: self.L00inv(l, self.Q(l)[:, 0] - self.L01SigT(l, z))))
        return F, z

    def rhs_lm(self):
        F, _ = self._lm_F()
        out = np.zeros((self.nx, 4))
        out[:, 0] = self.P0(F)
        out[:, 1:] = self.SigL10(F)
        return out

    def recover_lm(self, X):
        """eq-lm-step4: Psi0 and Phi1 from the reduced unknowns."""
        X = X.reshape(self.nx, 4)
        X0, X1 = X[:, 0], X[:, 1:]
        F, z = self._lm_F()
        Psi0 = np.stack(self._angles_map(
            lambda l: self.L00inv(l, self.M0(l, X0) + self.L01SigT(l, X1)))) + F
        Phi1 = self.B11inv(-self.SigL10(Psi0) + self.SigQ1())
        return Psi0, Phi1

    # ---------------------------------------------------------------- RLMDG (Section 3.3)
    def R(self, l, u0, alpha=None):
        """R_alpha Pi_0 for angle l: Legendre coefficients [n_x][3] of b1, b2, b3: ((h/2) delta_x, (h/2) delta_y,
        (h/2)^2 delta_xy); with alpha None this is the linear part R, otherwise R u0 + r_alpha.  delta_xy is 0
        except for the Q1-type reconstruction (``q1``): the upwind y-difference of the reconstructed x-slopes,
        over h inside and h/2 against d alpha/dx = 2 a1 / h on the y-inflow boundary row."""
        n, m, h, p = self.n, self.m, self.h, self.p
        U = u0.reshape(m, n)
        bw = np.zeros(m) if alpha is None else alpha[l, 0, :m, 0]
        be = np.zeros(m) if alpha is None else alpha[l, 1, :m, 0]
        bs = np.zeros(n) if alpha is None else alpha[l, 2, :n, 0]
        bn = np.zeros(n) if alpha is None else alpha[l, 3, :n, 0]
        if p.ox[l] > 0:
            left = np.concatenate([bw[:, None], U[:, :-1]], axis=1)
            sp = np.concatenate([np.full((m, 1), h / 2), np.full((m, n - 1), h)], axis=1)
            dx = (U - left) / sp
            if self.three_cell and n > 2:      # RLMDG*: quadratic through three upwind cell averages
                dx[:, 2:] = (3 * U[:, 2:] - 4 * U[:, 1:-1] + U[:, :-2]) / (2 * h)
        else:
            right = np.concatenate([U[:, 1:], be[:, None]], axis=1)
            sp = np.concatenate([np.full((m, n - 1), h), np.full((m, 1), h / 2)], axis=1)
            dx = (right - U) / sp
            if self.three_cell and n > 2:
                dx[:, :-2] = (-3 * U[:, :-2] + 4 * U[:, 1:-1] - U[:, 2:]) / (2 * h)
        if p.oy[l] > 0:
            down = np.concatenate([bs[None, :], U[:-1, :]], axis=0)
            sp = np.concatenate([np.full((1, n), h / 2), np.full((m - 1, n), h)], axis=0)
            dy = (U - down) / sp
            if self.three_cell and m > 2:
                dy[2:, :] = (3 * U[2:, :] - 4 * U[1:-1, :] + U[:-2, :]) / (2 * h)
        else:
            up = np.concatenate([U[1:, :], bn[None, :]], axis=0)
            sp = np.concatenate([np.full((m - 1, n), h), np.full((1, n), h / 2)], axis=0)
            dy = (up - U) / sp
            if self.three_cell and m > 2:
                dy[:-2, :] = (-3 * U[:-2, :] + 4 * U[1:-1, :] - U[2:, :]) / (2 * h)
        if self.supp is not None:
            bits = self.supp.reshape(m, n)
            dx = np.where(bits & (1 if p.ox[l] > 0 else 2), 0.0, dx)
            dy = np.where(bits & (4 if p.oy[l] > 0 else 8), 0.0, dy)
        dxy = np.zeros((m, n))
        if self.q1:
            if p.oy[l] > 0:
                gS = np.zeros(n) if alpha is None else 2.0 * alpha[l, 2, :n, 1] / h
                dxy = (dx - np.concatenate([gS[None, :], dx[:-1, :]], axis=0)) / \
                    np.concatenate([np.full((1, n), h / 2), np.full((m - 1, n), h)], axis=0)
            else:
                gN = np.zeros(n) if alpha is None else 2.0 * alpha[l, 3, :n, 1] / h
                dxy = (np.concatenate([dx[1:, :], gN[None, :]], axis=0) - dx) / \
                    np.concatenate([np.full((m - 1, n), h), np.full((1, n), h / 2)], axis=0)
        return np.stack([0.5 * h * dx.ravel(), 0.5 * h * dy.ravel(), 0.25 * h * h * dxy.ravel()], axis=1)

    def r_alpha(self, l):
        return self.R(l, np.zeros(self.nx), self.p.alpha) if self.p.alpha is not None else np.zeros((self.nx, 3))

    def P1(self, S):
        """P1 of a per-angle slope field S [n_Omega][n_x][k]: weighted angular sum."""
        return np.einsum("l,lkr->kr", self.p.w, S)

    def _slopes2(self, S2):
        """Cell functions with the reconstructed coefficients S2 [n_x][3] of b1, b2, b3."""
        u = np.zeros((self.nx, 4))
        u[:, 1:] = S2
        return u

    def SigLt10(self, Psi0, P1R=None):
        """Sigma Ltilde10 Psi0 = Sigma [L10 + L11 (I - Sigma^T P1) R] Psi0."""
        if P1R is None:
            P1R = self.P1(np.stack(self._angles_map(lambda l: self.R(l, Psi0[l]))))

        def one(l):
            u = self._const(Psi0[l])
            u[:, 1:] += self.R(l, Psi0[l]) - P1R
            return self.L(l, u)[:, 1:]
        return self._angles_sum(one, (self.nx, 3))

    def Gprime(self, Psi0):
        """Second block row operator: Sigma Ltilde10 + B11 P1 R."""
        P1R = self.P1(np.stack(self._angles_map(lambda l: self.R(l, Psi0[l]))))
        return self.SigLt10(Psi0, P1R) + self.B11fast(P1R)

    def _rlm_Qt(self):
        """Qtilde0 (per angle) and Sigma Qtilde1, with Qtilde_r = Q_r - L_r1 (I - Sigma^T P1) r_alpha."""
        ra = np.stack(self._angles_map(self.r_alpha))             # [n_Omega][n_x][3]
        P1ra = self.P1(ra)

        def qt(l):
            return self.Q(l) - self.L(l, self._slopes2(ra[l] - P1ra))
        Qt = self._angles_map(qt)
        return Qt

    def K_rlm(self, X):
        X = X.reshape(self.nx, 4)
        X0, X1 = X[:, 0], X[:, 1:]
        Psi0 = np.stack(self._angles_map(lambda l: self.Lt00inv(l, self.M0(l, X0) + self.L01SigT(l, X1))))
        out = np.zeros((self.nx, 4))
        out[:, 0] = X0 - self.P0(Psi0)
        out[:, 1:] = self.B11fast(X1) - self.Gprime(Psi0)
        return out

    def _rlm_F(self):
        Qt = self._rlm_Qt()
        SQt1 = np.zeros((self.nx, 3))
        for l in range(self.na):
            SQt1 += Qt[l][:, 1:]
        z = self.B11inv(SQt1)
        F = np.stack(self._angles_map(lambda l: self.Lt00inv(l, Qt[l][:, 0] - self.L01SigT(l, z))))
        return F, z, SQt1

    def rhs_rlm(self):
        F, _, _ = self._rlm_F()
        out = np.zeros((self.nx, 4))
        out[:, 0] = self.P0(F)
        out[:, 1:] = self.Gprime(F)
        return out

    def recover_rlm(self, X):
        X = X.reshape(self.nx, 4)
        X0, X1 = X[:, 0], X[:, 1:]
        F, z, SQt1 = self._rlm_F()
        Psi0 = np.stack(self._angles_map(
            lambda l: self.Lt00inv(l, self.M0(l, X0) + self.L01SigT(l, X1)))) + F
        Phi1 = self.B11inv(SQt1 - self.SigLt10(Psi0))
        return Psi0, Phi1

    def full_rlm(self, Psi0, Phi1):
        """Reconstructed angular flux psi + R*_alpha psi on V_h: [n_Omega][n_x][4]."""
        RR = np.stack(self._angles_map(lambda l: self.R(l, Psi0[l], self.p.alpha)))
        RR = RR - self.P1(RR)[None]
        out = np.zeros((self.na, self.nx, 4))
        out[:, :, 0] = Psi0
        out[:, :, 1:] = Phi1[None]
        out[:, :, 1:] += RR
        return out

    # ---------------------------------------------------------------- P0-DG (V_{h,0}, Section 3.1)
    def K_p0(self, X):
        """Piecewise-constant S_N-DG reduced to the cell-average scalar flux: X0 - P0 L00^-1 M0 X0 (the
        scheme of Section 2.1.1 on V_{h,0}); the slope entries of the 4-vector are carried by the identity."""
        X = X.reshape(self.nx, 4)
        Psi0 = np.stack(self._angles_map(lambda l: self.L00inv(l, self.M0(l, X[:, 0]))))
        out = X.copy()
        out[:, 0] = X[:, 0] - self.P0(Psi0)
        return out

    def rhs_p0(self):
        F = np.stack(self._angles_map(lambda l: self.L00inv(l, self.Q(l)[:, 0])))
        out = np.zeros((self.nx, 4))
        out[:, 0] = self.P0(F)
        return out

    def recover_p0(self, X):
        X0 = X.reshape(self.nx, 4)[:, 0]
        return np.stack(self._angles_map(lambda l: self.L00inv(l, self.M0(l, X0) + self.Q(l)[:, 0])))

    # ---------------------------------------------------------------- drivers
    def K(self, variant, X):
        return {"std": self.K_std, "lm": self.K_lm, "rlm": self.K_rlm, "p0": self.K_p0}[variant](X)

    def rhs(self, variant):
        return {"std": self.rhs_std, "lm": self.rhs_lm, "rlm": self.rhs_rlm, "p0": self.rhs_p0}[variant]()

    def dense_K(self, variant):
        """The reduced operator as a dense matrix (column j = K e_j); small meshes only."""
        n4 = 4 * self.nx
        cols = []
        for j in range(n4):
            e = np.zeros(n4)
            e[j] = 1.0
            cols.append(self.K(variant, e).ravel())
        return np.array(cols).T

    def solve(self, variant, tol=1e-12, restart=30, maxiter=20000, direct=None, x0=None, precond=None,
              dsa_cycles=None, mg=None):
        """Solve the reduced system and recover the solution.  Returns a dict like ``dense.solve`` plus
        ``X`` (reduced unknowns [n_x][4]) and ``iters``.

        ``precond='jacobi'`` (default for the low-memory variants) right-preconditions GMRES by
        diag(I, diag(B11))^-1, which leaves the residual of the original system unchanged; ``precond='dsa'``
        adds the diffusion correction of the cell averages (:mod:`oracle.dsa`) to it (to the identity for the
        standard scheme and P0-DG), solved exactly or (``dsa_cycles``) by that many multigrid V-cycles;
        ``precond='vdsa'`` is the vertex diffusion correction of :mod:`oracle.vdsa` (each scheme's own diffusion
        limit) after the Jacobi scaling, its solve exact or ``dsa_cycles`` V-cycles (``mg``: multigrid options);
        ``precond='bvdsa'`` the same correction added to the cell-block Jacobi step B^-1 v, B the diagonal blocks of
        K (:func:`oracle.vdsa.diagonal_blocks`)."""
        if precond is None:
            precond = "none" if variant in ("std", "p0") else "jacobi"
        b = self.rhs(variant).ravel()
        n4 = b.size
        if direct is None:
            direct = n4 <= 1024
        info = {"iters": 0}
        if direct:
            X = np.linalg.solve(self.dense_K(variant), b)
        else:
            D = np.ones((self.nx, 4))
            if variant not in ("std", "p0") and precond in ("jacobi", "dsa", "vdsa", "bvdsa"):
                D[:, 1:] = self.B11mat().diagonal().reshape(self.nx, 3)
            if precond in ("vdsa", "bvdsa"):
                from oracle.vdsa import VertexCorrection, diagonal_blocks
                blocks = diagonal_blocks(self, variant) if precond == "bvdsa" else None
                Minv = VertexCorrection(self.p, variant, None if variant == "std" else D[:, 1:], cycles=dsa_cycles,
                                        blocks=blocks, **(mg or {}))
            elif precond == "dsa":
                from oracle.dsa import DiffusionCorrection
                corr = DiffusionCorrection(self.p, cycles=dsa_cycles)
                Minv = lambda v: corr(v) / D.ravel()
            elif precond == "jacobi":
                Minv = lambda v: v / D.ravel()
            else:
                Minv = lambda v: v
            op = spla.LinearOperator((n4, n4), matvec=lambda v: self.K(variant, Minv(v)).ravel(),
                                     dtype=np.float64)
            cnt = [0]
            if x0 is not None and precond in ("dsa", "vdsa", "bvdsa"):
                raise ValueError("an initial guess is not supported with the diffusion correction")
            y0 = None if x0 is None else x0.ravel() * (1.0 if precond != "jacobi" else D.ravel())
            Y, ierr = spla.gmres(op, b, x0=y0, rtol=tol, atol=0.0, restart=restart, maxiter=maxiter,
                                 callback=lambda r: cnt.__setitem__(0, cnt[0] + 1), callback_type="pr_norm")
            X = Minv(Y)
            info["iters"] = cnt[0]
            info["gmres_info"] = ierr
        X = X.reshape(self.nx, 4)
        out = {"X": X, **info}
        if variant == "std":
            psi = self.recover_std(X)
        elif variant == "p0":
            Psi0 = self.recover_p0(X)
            psi = np.zeros((self.na, self.nx, 4))
            psi[:, :, 0] = Psi0
            out.update(psi0=Psi0)
        elif variant == "lm":
            Psi0, Phi1 = self.recover_lm(X)
            psi = np.zeros((self.na, self.nx, 4))
            psi[:, :, 0] = Psi0
            psi[:, :, 1:] = Phi1[None]
            out.update(psi0=Psi0, phi1=Phi1)
        else:
            Psi0, Phi1 = self.recover_rlm(X)
            psi = self.full_rlm(Psi0, Phi1)
            out.update(psi0=Psi0, phi1=Phi1)
        out["psi"] = psi
        out["phi"] = np.einsum("l,lkr->kr", self.p.w, psi)
        return out


def _b11_sparse(so):
    """B11 as a sparse matrix, assembled by probing the matrix-free B11 apply: cells of equal colour
    (i + 2 j) mod 5 share no stencil neighbourhood, so 5 colours x 3 slope components recover every entry."""
    import scipy.sparse as sp
    n, m, nx = so.n, so.m, so.nx
    jj, ii = np.divmod(np.arange(nx), n)
    col = (ii + 2 * jj) % 5
    nbrs = [np.arange(nx)]
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (ii + di >= 0) & (ii + di < n) & (jj + dj >= 0) & (jj + dj < m)
        nbrs.append(np.where(ok, (jj + dj) * n + ii + di, -1))
    rows, cols, vals = [], [], []
    for c in range(5):
        for s in range(3):
            e = np.zeros((nx, 3))
            e[col == c, s] = 1.0
            y = so.B11(e)                                # [nx][3]
            # column (K, s) for every K of colour c: entries live in K and its 4 neighbours
            for nb in nbrs:
                src = np.where(nb >= 0, nb, 0)
                mask = (nb >= 0) & (col == c)            # row cell = neighbour of a probed cell
                # row index: the neighbour cell nb[K]; column: probed cell K
                K = np.nonzero(mask)[0]
                R = nb[K]
                for r in range(3):
                    rows.append(3 * R + r)
                    cols.append(3 * K + s)
                    vals.append(y[R, r])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * nx, 3 * nx))
    A.sum_duplicates()
    return A


def adjoint_std(so, g, tol=1e-13, direct=None):
    """Sensitivities of J = sum_K g_K int_K psi_bar dx for the standard scheme (no paper counterpart: the
    discrete adjoint of eq-sndg-mat).  Per direction the state satisfies Lhat_l psi_l = Mhat Phi + Qhat_l; the
    multipliers satisfy Lhat_l^T lam_l = G + Mhat^T Lam, Lam = sum_l w_l lam_l, G_K = g_K int_K b_r (r = 0),
    solved through the reduced system Lam - sum_l w_l Lhat_l^-T Mhat Lam = sum_l w_l Lhat_l^-T G with the
    reverse transposed sweeps.  dJ/dp = sum_l w_l lam_l^T (dQhat_l/dp - dLhat_l/dp psi_l + dMhat/dp Phi):
      sigma_s: dLhat = dMhat = mass/eps;  sigma_a: dLhat = eps mass;  q (cell constant): dQhat = eps mass e_0.
    Returns (J, dJ/dsigma_s, dJ/dsigma_a, dJ/dq, lam, psi)."""
    p = so.p
    fwd = so.solve("std", tol=tol, direct=direct)
    psi, Phi = fwd["psi"], fwd["phi"]
    mass = so.mass
    G = np.zeros((so.nx, 4))
    G[:, 0] = g * mass[0, 0]
    J = float(np.sum(g * (Phi @ mass.T)[:, 0]))
    n4 = 4 * so.nx

    def Kadj(v):
        v = v.reshape(so.nx, 4)
        acc = so._angles_sum(lambda l: p.w[l] * so.LTinv(l, p.w[l] * so.sse[:, None] * (v @ mass.T)), (so.nx, 4))
        return (v - acc).ravel()
    b = so._angles_sum(lambda l: p.w[l] * so.LTinv(l, p.w[l] * G), (so.nx, 4)).ravel()
    if direct is None:
        direct = n4 <= 1024
    if direct:
        Km = np.array([Kadj(e) for e in np.eye(n4)]).T
        Lam = np.linalg.solve(Km, b).reshape(so.nx, 4)
    else:
        op = spla.LinearOperator((n4, n4), matvec=Kadj, dtype=np.float64)
        Lam, _ = spla.gmres(op, b, rtol=tol, atol=0.0, restart=30, maxiter=20000)
        Lam = Lam.reshape(so.nx, 4)
    MLam = so.sse[:, None] * (Lam @ mass.T)
    lam = np.stack(so._angles_map(lambda l: so.LTinv(l, p.w[l] * (G + MLam))))
    # weighted per-cell correlations sum_l w_l lam_l^T mass psi_l and Lam^T mass Phi
    corr = np.einsum("l,lkr,rs,lks->k", p.w, lam, mass, psi)
    lamPhi = np.einsum("kr,rs,ks->k", Lam, mass, Phi)
    d_ss = (lamPhi - corr) / p.eps
    d_sa = -p.eps * corr
    d_q = p.eps * mass[0, 0] * Lam[:, 0]
    return J, d_ss, d_sa, d_q, lam, psi

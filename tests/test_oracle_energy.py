"""Pin of the dense oracle by the energy identity behind the stability estimate eq-stab (Theorem
thm-gene-uni-solvency, Section 3.1).

For a Galerkin scheme (trial space = test space: Q1-DG on V_h, LMDG on V_h^lm, P0-DG on V_{h,0}) and vacuum inflow,
testing the discrete problem with the solution itself gives, term by term (upwind DG: every interior face
contributes half the squared jump of psi weighted by |Omega . n|, every boundary face half the squared trace),
    1/2 [[psi]]^2 + (1/eps) ||sigma_s^1/2 (psi - psi_bar)||^2 + eps ||sigma_a^1/2 psi||^2 = eps (q, psi),
with ||v||^2 = sum_j w_j int v_j^2 and [[psi]]^2 = sum_j w_j (sum over interior faces int |Omega_j . n| [psi_j]^2 +
sum over boundary faces int |Omega_j . n| psi_j^2).  Young's inequality on the right-hand side then gives eq-stab:
    (1/eps) ||sigma_s^1/2 (psi - psi_bar)||^2 + (eps/2) ||sigma_a^1/2 psi||^2 + 1/2 [[psi]]^2 <= eps/(2 delta_a) ||q||^2.
Every term here is computed from the oracle's solution coefficients with closed-form Legendre integrals (face
traces and the diagonal Q1 mass), independently of the oracle's assembled matrices, so a wrong factor in the
symmetric part of the assembly -- a face flux, the mass, the scattering weights -- breaks the identity (shown below
for the scattering weights).  Its antisymmetric part cancels in psi^T B psi; the sweep-equals-dense and exact-state
pins cover that part.
"""
import numpy as np
import pytest

from oracle import dense
from tests.helpers import random_problem

MASS = np.array([1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0])


def _face(a, b, h):
    """int over a face of length h of (a + b t)^2, t in [-1, 1] along the face."""
    return h * (a * a + b * b / 3.0)


def _energy_terms(p, psi):
    n, m, h = p.n, p.rows, p.h
    w, ox, oy = p.w, p.ox, p.oy
    U = psi.reshape(p.nang, m, n, 4)                       # [l][j][i][r]
    jump = 0.0
    for l in range(p.nang):
        u = U[l]
        east = (u[..., 0] + u[..., 1], u[..., 2] + u[..., 3])
        west = (u[..., 0] - u[..., 1], u[..., 2] - u[..., 3])
        north = (u[..., 0] + u[..., 2], u[..., 1] + u[..., 3])
        south = (u[..., 0] - u[..., 2], u[..., 1] - u[..., 3])
        a, b = abs(ox[l]), abs(oy[l])
        # interior vertical faces: east trace of (i) against west trace of (i + 1)
        s = _face(east[0][:, :-1] - west[0][:, 1:], east[1][:, :-1] - west[1][:, 1:], h).sum() * a
        s += _face(north[0][:-1, :] - south[0][1:, :], north[1][:-1, :] - south[1][1:, :], h).sum() * b
        # boundary faces (inflow and outflow alike: the inflow data is zero)
        s += (_face(west[0][:, 0], west[1][:, 0], h).sum() + _face(east[0][:, -1], east[1][:, -1], h).sum()) * a
        s += (_face(south[0][0, :], south[1][0, :], h).sum() + _face(north[0][-1, :], north[1][-1, :], h).sum()) * b
        jump += w[l] * s
    h2 = h * h
    psibar = np.einsum("l,lkr->kr", w, psi)
    dev = psi - psibar[None]
    scat = np.einsum("l,k,lkr,r->", w, p.sigma_s, dev * dev, MASS) * h2
    absn = np.einsum("l,k,lkr,r->", w, p.sigma_a, psi * psi, MASS) * h2
    q = p.q if p.q.ndim == 3 else np.broadcast_to(p.q, psi.shape)
    q_psi = np.einsum("l,lkr,lkr,r->", w, q, psi, MASS) * h2
    q_norm2 = np.einsum("l,lkr,r->", w, q * q, MASS) * h2
    return jump, scat, absn, q_psi, q_norm2


@pytest.mark.parametrize("variant", ["std", "lm", "p0"])
@pytest.mark.parametrize("eps", [1.0, 0.1, 1e-2])
@pytest.mark.parametrize("q_per_angle", [False, True])
def test_energy_identity_and_stability_estimate(variant, eps, q_per_angle):
    p = random_problem(3, 4, eps, 17, alpha=False, q_per_angle=q_per_angle, ny=4)
    psi = dense.solve(p, variant)["psi"]
    jump, scat, absn, q_psi, q_norm2 = _energy_terms(p, psi)
    lhs = 0.5 * jump + scat / eps + eps * absn
    rhs = eps * q_psi
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs), (lhs, rhs)
    delta_a = p.sigma_a.min()
    assert scat / eps + 0.5 * eps * absn + 0.5 * jump <= eps / (2.0 * delta_a) * q_norm2 * (1 + 1e-12)


@pytest.mark.parametrize("scale", [0.0, 0.95, 1.05])
def test_energy_identity_fails_for_a_wrong_scattering_weight(scale):
    """The identity separates the assembly from plausible mistakes in it: a scattering operator S with a wrong
    weight (scaled, or dropped) gives a solution whose energy terms no longer balance.  (A transposed B cannot
    serve as a negative case: psi^T B^T psi = psi^T B psi.)"""
    p = random_problem(3, 4, 1.0, 18, alpha=False, q_per_angle=False, ny=3)
    L, S, Q = dense.operator_matrices(p)
    psi = np.linalg.solve(L - scale * S, Q).reshape(p.nang, p.nx, 4)
    jump, scat, absn, q_psi, _ = _energy_terms(p, psi)
    lhs = 0.5 * jump + scat / p.eps + p.eps * absn
    assert abs(lhs - p.eps * q_psi) > 1e-3 * abs(p.eps * q_psi)

"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

* Appendix A building blocks against their closed forms, and the two oracles' integrals against each other.
* The sweep oracle (paper's block algorithms) against the dense brute-force solve on tiny meshes.
* States that lie in a trial space are reproduced exactly (constant and bilinear isotropic states for all
  variants, the anisotropic linear state for Q1-DG and RLMDG but not LMDG).
* Particle balance (test function v = 1, which lies in every test space).
* B11 symmetric positive definite (Theorem lem-B11) and the reduced operators nonsingular (Theorems
  thm-sndg-mat-psi and thm-K).
* Reduced-system dimensions of Table tab-compare and unknown counts of Table tab-sndg-costper.
* The RLMDG reduced system as printed does not reproduce the scheme; the corrected second row does.
"""
import copy

import numpy as np
import pytest

from oracle import dense
from oracle.sweeps import SweepOracle, elem_tables
from workloads.problems import mms_problem, uniform_problem, mms_sin, mms_aniso

VARIANTS = ("std", "lm", "rlm")


def test_elem_tables_closed_form():
    h = 0.37
    t = elem_tables(h)
    assert np.allclose(t["mass"], h * h * np.diag([1, 1 / 3, 1 / 3, 1 / 9]), atol=1e-15)
    vx = np.zeros((4, 4))
    vx[1, 0] = 2 * h          # int b0 d_x xi
    vx[3, 2] = 2 * h / 3      # int eta d_x (xi eta)
    vy = np.zeros((4, 4))
    vy[2, 0] = 2 * h
    vy[3, 1] = 2 * h / 3
    assert np.allclose(t["vol"][0], vx, atol=1e-15) and np.allclose(t["vol"][1], vy, atol=1e-15)
    # west face (xi = -1): traces (1, -1, eta, -eta); int over the face of length h
    tw = h / 2 * np.array([[2, -2, 0, 0], [-2, 2, 0, 0], [0, 0, 2 / 3, -2 / 3], [0, 0, -2 / 3, 2 / 3]])
    assert np.allclose(t["self"][0], tw, atol=1e-15)
    # neighbour across the west face sees its own east trace (1, 1, eta, eta)
    nw = h / 2 * np.array([[2, 2, 0, 0], [-2, -2, 0, 0], [0, 0, 2 / 3, 2 / 3], [0, 0, -2 / 3, -2 / 3]])
    assert np.allclose(t["nbr"][0], nw, atol=1e-15)
    m, vol, selfF, nbrF, _ = dense._ref_integrals(h)
    assert np.allclose(m, t["mass"], atol=1e-15) and np.allclose(vol, t["vol"], atol=1e-15)
    assert np.allclose(selfF, t["self"], atol=1e-15) and np.allclose(nbrF, t["nbr"], atol=1e-15)


def _random_problem(n, N, eps, seed, alpha=True):
    rng = np.random.default_rng(seed)
    p = uniform_problem(n, N, 1.0, 1.0, 1.0, eps=eps)
    p.sigma_s = rng.uniform(0.2, 3.0, p.nx)
    p.sigma_a = rng.uniform(0.1, 2.0, p.nx)
    p.q = rng.uniform(0.0, 2.0, (p.nang, p.nx, 4))
    if alpha:
        p.alpha = rng.uniform(0.0, 1.0, (p.nang, 4, n, 2))
    return p


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("eps", [1.0, 1e-2])
def test_sweep_oracle_equals_dense(variant, eps):
    p = _random_problem(3, 4, eps, 11)
    d = dense.solve(p, variant)
    s = SweepOracle(p).solve(variant, direct=True)
    scale = np.abs(d["psi"]).max()
    assert np.abs(d["psi"] - s["psi"]).max() <= 1e-11 * scale
    assert np.abs(d["phi"] - s["phi"]).max() <= 1e-11 * np.abs(d["phi"]).max()
    if variant != "std":
        assert np.abs(d["psi0"] - s["psi0"]).max() <= 1e-11 * scale


@pytest.mark.parametrize("variant", VARIANTS)
def test_sweep_oracle_equals_dense_rect_s8(variant):
    p = _random_problem(4, 8, 0.5, 12)
    d = dense.solve(p, variant)
    s = SweepOracle(p).solve(variant, direct=True)
    assert np.abs(d["psi"] - s["psi"]).max() <= 1e-11 * np.abs(d["psi"]).max()


_STATES = {
    "const": (lambda x, y, a, b: 0 * x + 2.5, lambda x, y, a, b: 0 * x, lambda x, y, a, b: 0 * x),
    "bilinear": (lambda x, y, a, b: 1 + 0.3 * x - 0.7 * y + 0.5 * x * y,
                 lambda x, y, a, b: 0.3 + 0.5 * y + 0 * x, lambda x, y, a, b: -0.7 + 0.5 * x + 0 * y),
    "aniso_linear": (lambda x, y, a, b: a * x + 0 * y, lambda x, y, a, b: a + 0 * x,
                     lambda x, y, a, b: 0 * x),
}


@pytest.mark.parametrize("state", list(_STATES))
@pytest.mark.parametrize("eps", [1.0, 0.1])
def test_exact_states(state, eps):
    f, fx, fy = _STATES[state]
    p = mms_problem(3, 4, f, fx, fy, sigma_s=1.0, sigma_a=0.5, eps=eps)
    so = SweepOracle(p)
    for v in VARIANTS:
        for res in (dense.solve(p, v), so.solve(v, direct=True)):
            err = np.abs(res["phi"][:, 0] - p.info["phi_avg"]).max()
            if state == "aniso_linear" and v == "lm":
                assert err > 1e-3, "LMDG cannot represent anisotropic slopes"
            else:
                assert err < 1e-12 * max(1.0, 1 / eps), (state, v, err)


def _balance(p, psi):
    """Particle balance terms for a full-space solution psi [n_Omega][n_x][4] (test function v = 1)."""
    n, h = p.n, p.h
    P = psi.reshape(p.nang, n, n, 4)
    leak = 0.0
    inflow = 0.0
    for l in range(p.nang):
        a, b = p.ox[l], p.oy[l]
        # face integrals of the traces: east h (c0 + c1), west h (c0 - c1), north h (c0 + c2), south h (c0 - c2)
        tr = {1: h * (P[l, :, -1, 0] + P[l, :, -1, 1]), 0: h * (P[l, :, 0, 0] - P[l, :, 0, 1]),
              3: h * (P[l, -1, :, 0] + P[l, -1, :, 2]), 2: h * (P[l, 0, :, 0] - P[l, 0, :, 2])}
        on = {0: -a, 1: a, 2: -b, 3: b}
        for side in range(4):
            if on[side] > 0:
                leak += p.w[l] * on[side] * tr[side].sum()
            elif p.alpha is not None:
                inflow += p.w[l] * (-on[side]) * h * p.alpha[l, side, :, 0].sum()
    phi0 = np.einsum("l,lk->k", p.w, psi[:, :, 0])
    absorb = (p.eps * p.sigma_a * phi0).sum() * h * h
    qbar = np.einsum("l,lk->k", p.w, p.q[:, :, 0]) if p.q.ndim == 3 else p.q[:, 0]
    src = (p.eps * qbar).sum() * h * h
    return leak + absorb, src + inflow


@pytest.mark.parametrize("variant", VARIANTS)
def test_particle_balance(variant):
    p = _random_problem(4, 4, 0.3, 5)
    s = SweepOracle(p).solve(variant, direct=True)
    lhs, rhs = _balance(p, s["psi"])
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_b11_spd_and_reduced_nonsingular():
    p = _random_problem(4, 4, 0.2, 7, alpha=False)
    so = SweepOracle(p)
    B = so.B11mat().toarray()
    assert np.abs(B - B.T).max() <= 1e-14 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    for v in VARIANTS:
        K = so.dense_K(v)
        assert K.shape == (4 * p.nx, 4 * p.nx)               # Table tab-compare: system dimension 4 n_x
        sv = np.linalg.svd(K, compute_uv=False)
        assert sv.min() > 1e-8 * sv.max()


def test_b11_appendix_c_form():
    # Appendix C: B11(u, v) = eps sigma_a (u, v) + sum over Omega_x > 0 directions of w |Omega.nu| [u][v] on
    # faces (x-faces for the x-part, likewise y), for centrally symmetric quadratures.  Check on a random
    # slope field through the bilinear form value X^T B11 X.
    p = _random_problem(4, 8, 0.4, 9, alpha=False)
    so = SweepOracle(p)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((p.nx, 3))
    val = X.ravel() @ so.B11(X).ravel()
    n, h = p.n, p.h
    U = X.reshape(n, n, 3)
    mass = h * h * np.array([1 / 3, 1 / 3, 1 / 9])
    ref = (p.eps * p.sigma_a.reshape(n, n)[..., None] * mass * U * U).sum()
    Ax = (p.w * p.ox * (p.ox > 0)).sum()
    Ay = (p.w * p.oy * (p.oy > 0)).sum()
    # jump of the slope part across an x-face between (i, j) and (i+1, j): trace on the left cell's east
    # face is c1 + c3 eta + c2 eta..., i.e. (c1) + (c2 + c3) eta; on the right cell's west face -c1 + (c2 - c3) eta
    for j in range(n):
        for i in range(n + 1):
            L = U[j, i - 1] if i > 0 else np.zeros(3)
            R = U[j, i] if i < n else np.zeros(3)
            m0 = L[0] + R[0]                      # constant part of [u] along the face
            m1 = (L[1] + L[2]) - (R[1] - R[2])    # eta part
            ref += Ax * h * (m0 * m0 + m1 * m1 / 3)
    for j in range(n + 1):
        for i in range(n):
            D = U[j - 1, i] if j > 0 else np.zeros(3)
            T = U[j, i] if j < n else np.zeros(3)
            m0 = D[1] + T[1]
            m1 = (D[0] + D[2]) - (T[0] - T[2])
            ref += Ay * h * (m0 * m0 + m1 * m1 / 3)
    assert abs(val - ref) <= 1e-12 * abs(ref)


def test_unknown_counts():
    # Table tab-sndg-costper (Q1, d = 2): standard 4 n_Omega per cell, low-memory (n_Omega - 1) + 4
    p = uniform_problem(3, 8, 1, 1, 1)
    assert dense.lm_basis(p).shape == (p.nang * p.nx * 4, p.nx * (p.nang - 1 + 4))
    assert dense.rlm_trial_basis(p).shape[1] == p.nx * (p.nang + 3)


def test_rlm_printed_system_is_not_the_scheme():
    """The reduced RLMDG operator as printed (second block row Sigma Ltilde10 instead of G') solves a
    different system; the corrected operator reproduces the dense Petrov-Galerkin solve."""
    p = _random_problem(3, 4, 1.0, 3, alpha=False)
    so = SweepOracle(p)
    d = dense.solve(p, "rlm")
    good = so.solve("rlm", direct=True)
    assert np.abs(good["psi0"] - d["psi0"]).max() < 1e-11 * np.abs(d["psi0"]).max()
    K_print = np.zeros((4 * p.nx, 4 * p.nx))
    b_print = np.zeros(4 * p.nx)
    F, z, _ = so._rlm_F()
    b_print[0::4] = so.P0(F)
    b_print.reshape(p.nx, 4)[:, 1:] = so.SigLt10(F)
    for j in range(4 * p.nx):
        e = np.zeros((p.nx, 4))
        e.ravel()[j] = 1.0
        X0, X1 = e[:, 0], e[:, 1:]
        Psi0 = np.stack([so.Lt00inv(l, so.M0(l, X0) + so.L01SigT(l, X1)) for l in range(p.nang)])
        col = np.zeros((p.nx, 4))
        col[:, 0] = X0 - so.P0(Psi0)
        col[:, 1:] = so.B11(X1) - so.SigLt10(Psi0)
        K_print[:, j] = col.ravel()
    Xp = np.linalg.solve(K_print, b_print).reshape(p.nx, 4)
    assert np.abs(Xp[:, 0] - good["X"][:, 0]).max() > 1e-6 * np.abs(good["X"][:, 0]).max()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_rectangular_mesh_transpose_symmetry_and_dense(variant):
    """Rectangular meshes (Section 2.1's mesh need not be square): the sweep oracle equals the dense one on a 3 x 5
    and a 1 x 4 mesh, and swapping the axes maps the 3 x 5 problem onto the 5 x 3 one (the level-symmetric set is
    invariant under Omega_x <-> Omega_y): cell (i, j) <-> (j, i), moments xi <-> eta, west/east <-> south/north
    inflow data.  A mix-up of the row and column counts anywhere breaks one of these."""
    from tests.helpers import random_problem
    for n, m in ((3, 5), (1, 4)):
        p = random_problem(n, 4, 0.6, 11, q_per_angle=False, ny=m)
        p.alpha = np.random.default_rng(12).uniform(0, 1, (1, 4, max(n, m), 2)).repeat(p.nang, axis=0)
        a = SweepOracle(p).solve(variant, direct=True)["phi"]
        assert np.abs(a - dense.solve(p, variant)["phi"]).max() <= 1e-13 * np.abs(a).max()
        t = copy.deepcopy(p)
        t.n, t.ny = m, n
        perm = np.arange(n * m).reshape(m, n).T.ravel()       # cell (j, i) of the transposed mesh
        t.sigma_s, t.sigma_a = p.sigma_s[perm], p.sigma_a[perm]
        t.q = p.q[perm][:, [0, 2, 1, 3]]
        t.alpha = p.alpha[:, [2, 3, 0, 1]]
        b = SweepOracle(t).solve(variant, direct=True)["phi"]
        assert np.abs(b[:, [0, 2, 1, 3]] - a[perm]).max() <= 1e-12 * np.abs(a).max()

"""Pins of the Q1-type reconstruction (Section 3.3.1 mentions it as converging alike and gives no formula).

Reading: besides the two-cell P1 slopes, the coefficient (h/2)^2 delta_xy of b3 = xi eta, delta_xy the upwind
y-difference of the reconstructed x-slopes (spacing h, and h/2 against the derivative 2 a1 / h of the inflow data
along the y-inflow boundary face).  Pins:

* the xi eta coefficient of the reconstruction of a bilinear function's cell averages (with its exact face data)
  is exactly its mixed derivative times (h/2)^2, in every cell and for every direction;
* with it RLMDG reproduces anisotropic bilinear states psi_l = c(Omega_l) x y exactly (the two-cell
  reconstruction does not), and isotropic and linear states stay exact;
* the sweep oracle equals the dense one (3 x 4 and 4 x 4 meshes, inflow data, eps 1 and 1e-2);
* the P1 slopes are those of the two-cell reconstruction, so the row-0 sweep is the same and only the slope rows
  of the reduced system change.
"""
import numpy as np
import pytest

from oracle import dense
from oracle.sweeps import SweepOracle
from tests.helpers import random_problem
from workloads.problems import mms_problem


def _bilinear_problem(n, N, c, d0=0.3, eps=0.7):
    return mms_problem(n, N, lambda x, y, a, b: c(a, b) * x * y + d0, lambda x, y, a, b: c(a, b) * y,
                       lambda x, y, a, b: c(a, b) * x, sigma_s=1.3, sigma_a=0.4, eps=eps)


def test_mixed_coefficient_exact_for_bilinear():
    n = 5
    p = _bilinear_problem(n, 4, lambda a, b: 1.0)
    X, Y = p.cell_centres()
    u0 = np.tile(X * Y + 0.3, (p.nang, 1))                 # cell averages of x y + 0.3 (exact: bilinear)
    R = dense.reconstruct(p, u0, p.alpha, q1=True)
    assert np.abs(R[:, :, 3] - (p.h / 2) ** 2).max() < 1e-14
    assert np.abs(R[:, :, 1] - (p.h / 2) * Y[None]).max() < 1e-14
    assert np.abs(R[:, :, 2] - (p.h / 2) * X[None]).max() < 1e-14
    R2 = dense.reconstruct(p, u0, p.alpha)
    assert np.array_equal(R2[:, :, 1:3], R[:, :, 1:3]) and not R2[:, :, 3].any()


@pytest.mark.parametrize("c", [lambda a, b: a, lambda a, b: (a - 2 * b) ** 2])
def test_anisotropic_bilinear_state_exact(c):
    p = _bilinear_problem(4, 4, c)
    exact = p.info["phi_avg"]
    q1 = dense.solve(p, "rlm", q1=True)["phi"][:, 0]
    two = dense.solve(p, "rlm")["phi"][:, 0]
    assert np.abs(q1 - exact).max() < 1e-13
    assert np.abs(two - exact).max() > 1e-7
    s = SweepOracle(p, q1=True).solve("rlm", direct=True)["phi"][:, 0]
    assert np.abs(s - exact).max() < 1e-13


def test_isotropic_linear_state_exact():
    p = mms_problem(4, 4, lambda x, y, a, b: 1 + 2 * x - y, lambda x, y, a, b: 2 + 0 * x,
                    lambda x, y, a, b: -1 + 0 * x, sigma_s=1.1, sigma_a=0.5, eps=0.5)
    r = dense.solve(p, "rlm", q1=True)["phi"][:, 0]
    assert np.abs(r - p.info["phi_avg"]).max() < 1e-13


@pytest.mark.parametrize("n,m,eps", [(3, 4, 1.0), (4, 4, 1e-2)])
def test_sweep_oracle_equals_dense(n, m, eps):
    p = random_problem(n, 4, eps, 31 + n, ny=m)
    d = dense.solve(p, "rlm", q1=True)
    s = SweepOracle(p, q1=True).solve("rlm", direct=True)
    assert np.abs(s["phi"] - d["phi"]).max() <= 1e-12 * np.abs(d["phi"]).max()
    assert np.abs(s["psi0"] - d["psi0"]).max() <= 1e-12 * np.abs(d["psi0"]).max()


def test_row0_sweep_unchanged():
    """The xi eta coefficient does not enter row 0 of any cell (its moment against b0 vanishes, on the cell and on
    every face), so the sweep for the cell averages is RLMDG's; the reduced operators differ in the slope rows."""
    p = random_problem(4, 4, 0.5, 41)
    a, b = SweepOracle(p), SweepOracle(p, q1=True)
    x = np.random.default_rng(2).standard_normal((p.nx, 4))
    ka, kb = a.K("rlm", x), b.K("rlm", x)
    assert np.array_equal(ka[:, 0], kb[:, 0])
    assert np.abs(ka[:, 1:] - kb[:, 1:]).max() > 1e-6 * np.abs(ka[:, 1:]).max()

"""Pins of the RLMDG variant without reconstruction across cross-section jumps (the remedy Section 4 gives for
the kinks at a discontinuity; the paper states no formula, the reading is that the upwind difference across an
interior face where (sigma_s, sigma_a) jumps is zero).

* In a homogeneous medium there is nothing to suppress: the variant is the RLMDG scheme itself.
* The dense Petrov-Galerkin solve and the sweep algorithm agree on media with many jumps.
* Exactness decides where suppression acts: the RLMDG trial space holds every isotropic linear function
  (the upwind differences of its cell averages are its slopes), so the scheme reproduces one exactly.  With
  suppression, a jump across x-faces removes the x-difference of the cells behind it for one half of the
  directions; the isotropic slope cannot then be matched in both halves, so a function linear in x is no
  longer reproduced, while one linear in y is (the y-differences are untouched); a jump across y-faces
  leaves functions linear in x exact.
"""
import numpy as np
import pytest

from oracle import dense
from oracle.sweeps import SweepOracle
from tests.helpers import random_problem
from workloads.problems import mms_problem


def _layered(axis, n=4, N=4, eps=1.0, slope_axis="x"):
    """Two media separated by the line axis = 0.5 (axis 'x': a jump across x-faces), psi = 0.3 + 0.7 t with
    t = x or y (isotropic)."""
    if axis == "x":
        ss = lambda x, y: np.where(x < 0.5, 1.0, 4.0)
        sa = lambda x, y: np.where(x < 0.5, 0.5, 0.2)
    else:
        ss = lambda x, y: np.where(y < 0.5, 1.0, 4.0)
        sa = lambda x, y: np.where(y < 0.5, 0.5, 0.2)
    if slope_axis == "x":
        f, fx, fy = (lambda x, y, a, b: 0.3 + 0.7 * x + 0 * y, lambda x, y, a, b: 0.7 + 0 * x,
                     lambda x, y, a, b: 0 * x)
    else:
        f, fx, fy = (lambda x, y, a, b: 0.3 + 0.7 * y + 0 * x, lambda x, y, a, b: 0 * x,
                     lambda x, y, a, b: 0.7 + 0 * y)
    return mms_problem(n, N, f, fx, fy, sigma_s=ss, sigma_a=sa, eps=eps)


def _err(p, res):
    return float(np.abs(res["phi"][:, 0] - p.info["phi_avg"]).max())


def test_homogeneous_medium_is_rlmdg():
    p = random_problem(4, 4, 1.0, 3)
    p.sigma_s[:] = 1.3
    p.sigma_a[:] = 0.4
    a, b = dense.solve(p, "rlm"), dense.solve(p, "rlm", suppress=True)
    assert np.array_equal(a["psi"], b["psi"])
    sa = SweepOracle(p).solve("rlm", direct=True)
    sb = SweepOracle(p, suppress=True).solve("rlm", direct=True)
    assert np.array_equal(sa["X"], sb["X"])


@pytest.mark.parametrize("eps", [1.0, 0.1])
def test_sweep_equals_dense_with_jumps(eps):
    # two materials in a random pattern: most interior faces are jumps
    p = random_problem(4, 4, eps, 11)
    rng = np.random.default_rng(5)
    pick = rng.integers(0, 2, p.nx)
    p.sigma_s = np.where(pick == 1, 2.0, 0.7)
    p.sigma_a = np.where(pick == 1, 0.3, 1.1)
    d = dense.solve(p, "rlm", suppress=True)
    s = SweepOracle(p, suppress=True).solve("rlm", direct=True)
    assert np.abs(s["phi"] - d["phi"]).max() <= 1e-12 * np.abs(d["phi"]).max()
    assert np.abs(s["psi"] - d["psi"]).max() <= 1e-12 * np.abs(d["psi"]).max()
    # suppression changes the answer on this medium
    assert np.abs(dense.solve(p, "rlm")["phi"] - d["phi"]).max() > 1e-6


@pytest.mark.parametrize("eps", [1.0, 0.1])
def test_jump_across_y_faces_keeps_x_linear_exact(eps):
    p = _layered("y", eps=eps, slope_axis="x")
    tol = 1e-12 * max(1.0, 1 / eps)
    for res in (dense.solve(p, "rlm", suppress=True), SweepOracle(p, suppress=True).solve("rlm", direct=True),
                dense.solve(p, "rlm")):
        assert _err(p, res) < tol


@pytest.mark.parametrize("eps", [1.0, 0.1])
def test_jump_across_x_faces(eps):
    tol = 1e-12 * max(1.0, 1 / eps)
    p = _layered("x", eps=eps, slope_axis="x")
    assert _err(p, dense.solve(p, "rlm")) < tol                 # plain RLMDG: exact
    for res in (dense.solve(p, "rlm", suppress=True), SweepOracle(p, suppress=True).solve("rlm", direct=True)):
        assert _err(p, res) > 1e-6                             # the suppressed x-difference shows
    p = _layered("x", eps=eps, slope_axis="y")
    for res in (dense.solve(p, "rlm", suppress=True), SweepOracle(p, suppress=True).solve("rlm", direct=True)):
        assert _err(p, res) < tol

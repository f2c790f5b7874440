"""Pins of P0-DG (the S_N-DG scheme of Section 2.1.1 on the piecewise constants V_{h,0}, the comparison scheme
of Section 3.1 and of the 1D tests, here in 2D).

* Dense Galerkin solve on V_{h,0} and the sweep algorithm (L00 sweeps, cell-average reduced system) agree.
* A constant isotropic state with its own source and inflow is reproduced exactly.
* First-order accuracy on the fabricated solution sin(x + y).
* Section 3.1: with piecewise constants the diffusion limit degenerates to a global constant (zero under
  vacuum inflow): the P0-DG scalar flux vanishes like eps, while LMDG keeps a finite diffusion limit.
"""
import numpy as np

from oracle import dense
from oracle.sweeps import SweepOracle
from tests.helpers import random_problem
from workloads.problems import mms_problem, mms_sin, uniform_problem


def test_sweep_equals_dense():
    for n, eps in ((3, 1.0), (4, 0.5)):
        p = random_problem(n, 4, eps, 3)
        d = dense.solve(p, "p0")
        s = SweepOracle(p).solve("p0", direct=True)
        assert np.abs(s["psi"] - d["psi"]).max() <= 1e-12 * np.abs(d["psi"]).max()


def test_constant_state_exact():
    p = mms_problem(4, 4, lambda x, y, a, b: 0.7 + 0 * x, lambda x, y, a, b: 0 * x, lambda x, y, a, b: 0 * x,
                    sigma_s=1.0, sigma_a=0.5, eps=0.3)
    for res in (dense.solve(p, "p0"), SweepOracle(p).solve("p0", direct=True)):
        assert np.abs(res["phi"][:, 0] - p.info["phi_avg"]).max() < 1e-12


def test_first_order():
    err = []
    for n in (8, 16, 32):
        p = mms_sin(n, 4)
        r = SweepOracle(p).solve("p0", direct=False, tol=1e-12)
        err.append(np.abs(r["phi"][:, 0] - p.info["phi_avg"]).mean())
    order = np.log2(err[1] / err[2])
    assert 0.8 < order < 1.2, err


def test_diffusion_limit_degenerates():
    mean = {}
    for eps in (1e-3, 1e-4):
        p = uniform_problem(6, 4, 1.0, 1.0, 1.0, eps=eps)
        mean[eps] = dense.solve(p, "p0")["phi"][:, 0].mean()
        lm = dense.solve(p, "lm")["phi"][:, 0].mean()
        assert lm > 0.05
    assert abs(mean[1e-3] / mean[1e-4] - 10.0) < 0.5
    assert mean[1e-4] < 1e-3

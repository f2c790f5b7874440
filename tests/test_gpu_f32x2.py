"""Float-float sweeps (LMDG_SWEEP_F32X2, the residual sweeps of the mixed solve with LMDG_RESID_F32X2) against
the oracle.

Tolerance.  Each float-float operation errs by a few units of 2^-48 of its operands where FP64 errs by 2^-53;
the FP64 sweeps are held to 1e-12, so the float-float ones are held to 2^5 times that, 3e-11.  Cases: every
scheme (Q1-DG, LMDG, RLMDG, RLMDG*, RLMDG with suppression, P0-DG), homogeneous and source (residual) mode
with angle-dependent sources and inflow data, one cell to ragged multi-strip meshes; mixed solves whose
residuals are float-float reach the FP64 solution; the adjoint through such solves.
"""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle, adjoint_std
from tests.helpers import random_problem, rel

pytestmark = pytest.mark.gpu

TOL_F2 = 3e-11


def _bprime(so, variant):
    b = so.rhs(variant)
    if variant in ("std", "p0"):
        return b
    z = so._lm_F()[1] if variant == "lm" else so._rlm_F()[1]
    e = np.zeros((so.nx, 4))
    e[:, 1:] = z
    return b - so.K(variant, e)


SCHEMES = [("std", {}, {}), ("lm", {}, {}), ("rlm", {}, {}), ("p0", {}, {}),
           ("rlm", {"recon": 1}, {"three_cell": True}), ("rlm", {"suppress": 1}, {"suppress": True})]


@pytest.mark.parametrize("scheme", range(len(SCHEMES)))
@pytest.mark.parametrize("n,N,eps,seed", [(1, 4, 1.0, 1), (5, 4, 1.0, 2), (37, 4, 1e-2, 3), (70, 8, 0.3, 4)])
def test_operator_apply(scheme, n, N, eps, seed):
    from paper_1907_01027_gb300 import Context, SWEEP_F32X2, SWEEP_SOURCE
    variant, copts, oopts = SCHEMES[scheme]
    if copts.get("recon") and n < 2:
        pytest.skip("RLMDG* on one cell is RLMDG")
    p = random_problem(n, N, eps, seed)
    if copts.get("suppress"):
        # two materials on 4x4-cell patches, so that the suppression bits are set across faces
        m = np.kron(np.random.default_rng(seed + 50).integers(0, 2, (-(-n // 4),) * 2), np.ones((4, 4), int))
        m = m[:n, :n].ravel()
        p.sigma_s = np.where(m == 1, 2.0, 0.7)
        p.sigma_a = np.where(m == 1, 0.3, 1.1)
    so = SweepOracle(p, **oopts)
    ctx = Context(p, variant, **copts)
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    ref = so.K(variant, x)
    assert rel(ctx.sweep(x, flags=SWEEP_F32X2), ref) < TOL_F2
    assert rel(ctx.sweep(x, flags=SWEEP_F32X2 | SWEEP_SOURCE), ref - _bprime(so, variant)) < TOL_F2
    ctx.close()


def test_flags_rejected():
    from paper_1907_01027_gb300 import Context, LmdgError, SWEEP_F32X2, SWEEP_FP32, SWEEP_STORE
    p = random_problem(6, 4, 1.0, 9)
    ctx = Context(p, "lm")
    x = np.zeros((p.nx, 4))
    for f in (SWEEP_F32X2 | SWEEP_STORE, SWEEP_F32X2 | SWEEP_FP32):
        with pytest.raises(LmdgError) as e:
            ctx.sweep(x, flags=f)
        assert e.value.code == -1
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm", "p0"])
@pytest.mark.parametrize("n,N,eps,seed", [(9, 4, 1.0, 21), (33, 8, 1.0, 23)])
def test_mixed_solve_with_f32x2_residuals(variant, n, N, eps, seed):
    from paper_1907_01027_gb300 import Context, FP32, RESID_F32X2
    p = random_problem(n, N, eps, seed)
    ref = SweepOracle(p).solve(variant, direct=True)
    ctx = Context(p, variant, precision=FP32, resid=RESID_F32X2, tol=1e-12, max_iters=20000)
    _, phi, st, rc = ctx.solve(exact_ref=True)
    assert rc == 0, st
    assert st["sweeps_fp64"] == 0 and st["sweeps_f32x2"] >= 1
    assert st["resid"] <= 1e-12 * st["resid0"]
    # with LMDG_SOLVE_EXACT_REF the tolerance reference ||b|| comes from a float-float sweep; without it, from an
    # FP32 sweep, within the FP32 sweep's error of the exact norm
    from paper_1907_01027_gb300 import SWEEP_SOURCE
    bn = np.linalg.norm(ctx.sweep(np.zeros((p.nx, 4)), flags=SWEEP_SOURCE))
    assert abs(st["resid0"] - bn) <= 1e-12 * bn, (st["resid0"], bn)
    _, _, st32, rc32 = ctx.solve()
    assert rc32 == 0 and abs(st32["resid0"] - bn) <= 1e-5 * bn, (st32["resid0"], bn)
    # kappa * tol: the reduced operators at these sizes have kappa of order 1 / h^2 ~ 1e3
    assert rel(phi, ref["phi"]) < 1e-8
    ctx.close()


def test_mixed_adjoint_with_f32x2_residuals():
    from paper_1907_01027_gb300 import Context, FP32, RESID_F32X2
    p = random_problem(12, 8, 0.6, 91, q_per_angle=False)
    g = np.random.default_rng(92).uniform(0, 1, p.nx)
    J0, a0, b0, c0, _, _ = adjoint_std(SweepOracle(p), g, direct=True)
    ctx = Context(p, "std", precision=FP32, resid=RESID_F32X2, tol=1e-12, max_iters=20000)
    J, dss, dsa, dq, st = ctx.adjoint(g)
    # as for the mixed adjoint with FP64 residuals: J to the solve tolerance, gradients to 1e-5
    assert abs(J - J0) <= 1e-9 * abs(J0)
    assert rel(dss, a0) < 1e-5 and rel(dsa, b0) < 1e-5 and rel(dq, c0) < 1e-5
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm", "p0"])
@pytest.mark.parametrize("n,N,eps,seed", [(5, 4, 1.0, 31), (70, 8, 0.3, 32)])
def test_source_sweep_vacuum_isotropic(variant, n, N, eps, seed):
    """Vacuum inflow and an isotropic source: the residual sweeps of such problems (the benchmark's) run the lean
    instances in FP32 and float-float."""
    from paper_1907_01027_gb300 import Context, SWEEP_F32X2, SWEEP_FP32, SWEEP_SOURCE
    p = random_problem(n, N, eps, seed, alpha=False, q_per_angle=False)
    so = SweepOracle(p)
    ctx = Context(p, variant)
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    ref = so.K(variant, x) - _bprime(so, variant)
    assert rel(ctx.sweep(x, flags=SWEEP_F32X2 | SWEEP_SOURCE), ref) < TOL_F2
    assert rel(ctx.sweep(x, flags=SWEEP_SOURCE), ref) < 1e-12
    assert rel(ctx.sweep(x, flags=SWEEP_FP32 | SWEEP_SOURCE), ref) < 1e-5
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_mixed_solve_vacuum_isotropic(variant):
    from paper_1907_01027_gb300 import Context, FP32, RESID_F32X2
    p = random_problem(16, 4, 1.0, 33, alpha=False, q_per_angle=False)
    ref = SweepOracle(p).solve(variant, direct=True)
    ctx = Context(p, variant, precision=FP32, resid=RESID_F32X2, tol=1e-12, max_iters=20000)
    _, phi, st, rc = ctx.solve()
    assert rc == 0 and st["sweeps_f32x2"] >= 1, st
    assert rel(phi, ref["phi"]) < 1e-8
    ctx.close()

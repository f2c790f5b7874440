"""GPU parity: the CUDA path through the C ABI against the FP64 oracle (element by element).

Tolerances: FP64 operator applications and source residuals 1e-12 relative (max norm); FP64 solves driven
to 1e-13 compared with the oracle's direct solve at 1e-10 (condition number times the stopping tolerance);
FP32 sweeps 1e-5 of the FP64 sweep at eps = 1; mixed-precision solves reach the FP64 residual target.
"""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import random_problem, rel

pytestmark = pytest.mark.gpu

VARIANTS = ("std", "lm", "rlm")


def _ctx(p, variant, **kw):
    from paper_1907_01027_gb300 import Context
    return Context(p, variant, **kw)


def _oracle_bprime(so, variant):
    """b' = b - K [0; z] (the right-hand side of the system lmdg_sweep's source mode zeroes)."""
    b = so.rhs(variant)
    if variant == "std":
        return b
    z = so._lm_F()[1] if variant == "lm" else so._rlm_F()[1]
    e = np.zeros((so.nx, 4))
    e[:, 1:] = z
    return b - so.K(variant, e)


CASES = [(5, 4, 1.0, 1), (37, 4, 1.0, 2), (37, 4, 1e-2, 3), (70, 4, 0.3, 4), (40, 8, 1.0, 5)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,N,eps,seed", CASES)
def test_operator_apply_fp64(variant, n, N, eps, seed):
    from paper_1907_01027_gb300 import SWEEP_SOURCE
    p = random_problem(n, N, eps, seed)
    so = SweepOracle(p)
    ctx = _ctx(p, variant)
    x = np.random.default_rng(seed + 100).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    ref = so.K(variant, x)
    assert rel(y, ref) < 1e-12
    ys = ctx.sweep(x, flags=SWEEP_SOURCE)
    refs = ref - _oracle_bprime(so, variant)
    assert rel(ys, refs) < 1e-12
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_isotropic_source_vacuum(variant):
    from paper_1907_01027_gb300 import SWEEP_SOURCE
    p = random_problem(45, 8, 1.0, 9, alpha=False, q_per_angle=False)
    so = SweepOracle(p)
    ctx = _ctx(p, variant)
    x = np.zeros((p.nx, 4))
    ys = ctx.sweep(x, flags=SWEEP_SOURCE)
    assert rel(ys, -_oracle_bprime(so, variant)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,N,eps,seed", [(9, 4, 1.0, 21), (16, 4, 0.1, 22), (12, 8, 1.0, 23)])
def test_solve_fp64_matches_oracle(variant, n, N, eps, seed):
    p = random_problem(n, N, eps, seed)
    so = SweepOracle(p)
    ref = so.solve(variant, direct=True)
    ctx = _ctx(p, variant, tol=1e-13, max_iters=20000)
    x, phi, st, rc = ctx.solve()
    assert rc == 0, st
    assert rel(phi, ref["phi"]) < 1e-10, st
    psi = ctx.get_psi()
    if variant == "std":
        assert rel(psi, ref["psi"]) < 1e-10
    else:
        assert rel(psi, ref["psi0"]) < 1e-10
        assert rel(phi[:, 1:], ref["phi1"]) < 1e-9
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_fp32_sweep_close_to_fp64(variant):
    from paper_1907_01027_gb300 import SWEEP_FP32, SWEEP_SOURCE
    p = random_problem(64, 8, 1.0, 31)
    ctx = _ctx(p, variant)
    x = np.random.default_rng(7).standard_normal((p.nx, 4))
    for fl in (0, SWEEP_SOURCE):
        y64 = ctx.sweep(x, flags=fl)
        y32 = ctx.sweep(x, flags=fl | SWEEP_FP32)
        assert rel(y32, y64) < 1e-5
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_solve(variant, prec):
    p = random_problem(16, 8, 1.0, 41)
    so = SweepOracle(p)
    ref = so.solve(variant, direct=True)
    # FP64-refined residual 1e-12 against the oracle's direct solve: error <= kappa * tol, kappa <= 1e4
    ctx = _ctx(p, variant, precision=prec, tol=1e-12)
    x, phi, st, rc = ctx.solve()
    assert rc == 0 and st["resid"] <= 1e-12 * st["resid0"], st
    assert st["sweeps_fp32"] > st["sweeps_fp64"], st
    assert rel(phi, ref["phi"]) < 1e-8
    psi = ctx.get_psi()
    tol = 1e-5 if prec == 1 else 1e-2
    assert rel(psi, ref["psi"] if variant == "std" else ref["psi0"]) < tol
    ctx.close()


def test_b11_apply_and_cg():
    p = random_problem(20, 8, 0.5, 51)
    so = SweepOracle(p)
    ctx = _ctx(p, "lm")
    X1 = np.random.default_rng(3).standard_normal((p.nx, 3))
    assert rel(ctx.b11_apply(X1), so.B11(X1)) < 1e-13
    r = so.SigQ1()
    z, it = ctx.b11_solve(r, tol=1e-14)
    assert rel(z, so.B11inv(r)) < 1e-10 and it > 0
    ctx.close()


def test_deterministic():
    p = random_problem(70, 8, 1.0, 61)
    for v in VARIANTS:
        ctx = _ctx(p, v)
        x = np.random.default_rng(5).standard_normal((p.nx, 4))
        a = ctx.sweep(x)
        b = ctx.sweep(x)
        assert np.array_equal(a, b)
        ctx.close()


def test_spin_limit_reports_timeout_and_context_survives():
    from paper_1907_01027_gb300 import LmdgError
    p = random_problem(256, 4, 1.0, 71, alpha=False, q_per_angle=False)
    ctx = _ctx(p, "lm", spin_limit=1)
    with pytest.raises(LmdgError) as ei:
        ctx.sweep(np.ones((p.nx, 4)))
    assert ei.value.code == -6
    ctx.close()
    ok = _ctx(p, "lm")
    y = ok.sweep(np.ones((p.nx, 4)))
    assert np.all(np.isfinite(y))
    ok.close()


@pytest.mark.parametrize("n", [37, 70])
def test_storing_sweep_psi_multistrip(n):
    """A storing source sweep keeps psi_l = L^-1 (M Phi + Q) (the recovery of eq-sndg-final-sweep) on meshes of
    two and three 32-row strips with a ragged last one, FP64 and FP32, read back in the user layout."""
    from paper_1907_01027_gb300 import SWEEP_FP32, SWEEP_SOURCE, SWEEP_STORE
    p = random_problem(n, 4, 1.0, 60 + n)
    so = SweepOracle(p)
    ctx = _ctx(p, "std")
    x = np.random.default_rng(n).standard_normal((p.nx, 4))
    ref = so.recover_std(x)
    ctx.sweep(x, flags=SWEEP_SOURCE | SWEEP_STORE)
    assert rel(ctx.get_psi(), ref) < 1e-12
    ctx.sweep(x, flags=SWEEP_SOURCE | SWEEP_STORE | SWEEP_FP32)
    assert rel(ctx.get_psi(), ref) < 1e-5
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_kappa_estimate_from_the_hessenberg(variant):
    """lmdg_stats.kappa_est, the condition number of a GMRES cycle's Hessenberg matrix, is a lower estimate of the
    condition number of the (here unpreconditioned) reduced operator, from the oracle's dense operator, and reaches
    it as the Krylov space fills (100 unknowns, one cycle of up to 100 iterations driven to stagnation)."""
    p = random_problem(5, 4, 0.3, 71, alpha=False, q_per_angle=False)
    so = SweepOracle(p)
    n = 4 * p.nx
    K = np.stack([so.K(variant, e.reshape(p.nx, 4)).ravel() for e in np.eye(n)], axis=1)
    cond = np.linalg.cond(K)
    ctx = _ctx(p, variant, precond=0, restart=n, tol=1e-15, max_iters=n)
    _, _, st, _ = ctx.solve(allow_stall=True)
    ctx.close()
    assert st["kappa_est"] <= cond * (1 + 1e-6), (st["kappa_est"], cond)
    assert st["kappa_est"] >= 0.5 * cond, (st["kappa_est"], cond, st["iters"])

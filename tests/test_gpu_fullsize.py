"""Parity at the benchmark's own sizes, in the launch configuration the benchmark uses.

* FP64 reduced-operator applications of all three schemes at 1024^2 cells, S16 (the benchmark workload), every
  output against the oracle at 1e-12 (the oracle applies B11 literally instead of assembling it).
* Source (residual) mode at 256^2, S8 (eps = 1e-2) against the oracle's right-hand side.
* FP32 against FP64 sweeps at 1024^2 (a property: agreement to FP32 accuracy), float-float sweeps against the
  oracle at 3e-11, and the mixed-precision solve against the FP64 solve on the 256^2 workload.
"""
import numpy as np
import pytest

from oracle.sweeps import SweepOracle
from tests.helpers import rel
from workloads.problems import config2, config4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg4():
    return config4(eps=1.0)


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_operator_apply_1024_s16(cfg4, variant):
    from paper_1907_01027_gb300 import Context, SWEEP_FP32, SWEEP_F32X2
    p = cfg4
    ctx = Context(p, variant)
    x = np.random.default_rng(7).standard_normal((p.nx, 4))
    y = ctx.sweep(x)
    so = SweepOracle(p, literal_b11=True)
    ref = so.K(variant, x)
    assert rel(y, ref) < 1e-12
    y32 = ctx.sweep(x, flags=SWEEP_FP32)
    assert rel(y32, y) < 1e-5
    # float-float (the residual sweeps of the mixed solve with LMDG_RESID_F32X2), against the oracle
    assert rel(ctx.sweep(x, flags=SWEEP_F32X2), ref) < 3e-11
    ctx.close()


def _bprime(so, variant):
    b = so.rhs(variant)
    if variant == "std":
        return b
    z = so._lm_F()[1] if variant == "lm" else so._rlm_F()[1]
    e = np.zeros((so.nx, 4))
    e[:, 1:] = z
    return b - so.K(variant, e)


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_source_mode_256_s8(variant):
    from paper_1907_01027_gb300 import Context, SWEEP_SOURCE
    p = config2(eps=1e-2)
    ctx = Context(p, variant)
    x = np.random.default_rng(8).standard_normal((p.nx, 4))
    y = ctx.sweep(x, flags=SWEEP_SOURCE)
    so = SweepOracle(p)
    ref = so.K(variant, x) - _bprime(so, variant)
    assert rel(y, ref) < 1e-12
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
def test_mixed_solve_matches_fp64_solve_256(variant):
    from paper_1907_01027_gb300 import Context
    # both solves to 1e-13: their difference is bounded by kappa * tol, and the low-memory operators, whose X1
    # rows are O(h) against O(1) X0 rows, have kappa ~ 1/h^2 ~ 6.5e4 at 256^2
    p = config2(eps=1.0)
    c64 = Context(p, variant, tol=1e-13, max_iters=20000)
    _, phi64, st64, rc64 = c64.solve()
    c64.close()
    c32 = Context(p, variant, tol=1e-13, precision=1, max_iters=20000)
    _, phi32, st32, rc32 = c32.solve()
    c32.close()
    assert rc64 == 0 and rc32 == 0
    assert st32["resid"] <= 1e-13 * st32["resid0"]
    assert rel(phi32, phi64) < 1e-7

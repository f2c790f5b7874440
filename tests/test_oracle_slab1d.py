"""Pins of the slab-geometry oracle (oracle/slab1d.py) against what the paper prints and the mathematics fixes.

* Table tab-1d-eps10-5 (Example examp-1ddifflim): every printed error of P0-DG, P1-DG, LMDG and RLMDG at
  eps = 1e-5 and 1, against the printed P1-DG reference on 1280 cells -- within 0.6% on 20 and 40 cells (three
  printed digits) and 5% on 80 and 160 (where the reference's own error enters); P0-DG's missing diffusion
  limit (error 2 = the L1 norm of the limit solution sin x).
* Table tab-1d-aniso (Example examp-1dfab): the printed observed orders to +-0.02, and the errors within 6% when
  the printed h is read as half the cell width (the reading that matches; it is listed among the readings).
* RLMDG* (the three-cell reconstruction, discussion of Example examp-1dfab): second order, error comparable
  to P1-DG's and well below RLMDG's, as the paper states.
* Exact states: constant isotropic psi for every scheme; linear isotropic psi for P1-DG, LMDG and RLMDG;
  the anisotropic linear psi = mu x for P1-DG and RLMDG but not LMDG (upwind differences and the inflow
  difference over h/2 are exact on linears); all to round-off.
"""
import os

import numpy as np
import pytest

from oracle.slab1d import Slab, diffusion_limit, fabricated, gauss_ordinates

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].split()
        if line:
            out.append(line)
    return out


def test_gauss_ordinates_moments():
    mu, w = gauss_ordinates(32)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(64):
        exact = 1.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * mu ** k) - exact) < 1e-14
    assert np.allclose(np.sort(mu), -np.sort(mu)[::-1], atol=1e-15)


@pytest.fixture(scope="module")
def diffusion_errors():
    out = {}
    for eps in (1e-5, 1.0):
        ref = diffusion_limit(1280, eps)
        cref = ref.solve("p1")
        for scheme in ("p0", "p1", "lm", "rlm"):
            for n in (20, 40, 80, 160):
                s = diffusion_limit(n, eps)
                out[(eps, scheme, n)] = s.l1_diff(s.solve(scheme), ref, cref)
    return out


def test_diffusion_table_reproduced(diffusion_errors):
    for eps, scheme, n, err in _rows("tab_1d_eps.txt"):
        ours = diffusion_errors[(float(eps), scheme, int(n))]
        tol = 0.006 if int(n) <= 40 else 0.05
        assert abs(ours / float(err) - 1.0) <= tol, (eps, scheme, n, ours, err)


def test_diffusion_limit_orders(diffusion_errors):
    e = diffusion_errors
    order = lambda eps, s, n: np.log2(e[(eps, s, n)] / e[(eps, s, 2 * n)])
    for n in (20, 40, 80):
        assert e[(1e-5, "p0", n)] > 1.9                       # no diffusion limit: phi_h ~ 0 against sin x
        for s in ("p1", "lm", "rlm"):
            assert abs(order(1e-5, s, n) - 2.0) < 0.1          # second order in the thick regime
        assert abs(order(1.0, "lm", n) - 1.0) < 0.1           # LMDG first order when psi is anisotropic
        assert abs(order(1.0, "p0", n) - 1.0) < 0.1
    for s in ("p1", "rlm"):
        assert order(1.0, s, 80) > 1.85


@pytest.fixture(scope="module")
def fabricated_errors():
    out = {}
    for case in ("iso", "aniso"):
        for scheme in ("p0", "p1", "lm", "rlm", "rlm3"):
            for k, n in enumerate((40, 80, 160, 320)):
                s, psi = fabricated(n, case)
                out[(case, scheme, k)] = s.l1_error(s.solve(scheme), psi)
    return out


def test_fabricated_table(fabricated_errors):
    hs = ("1/20", "1/40", "1/80", "1/160")
    for case, scheme, h, err, order in _rows("tab_1d_aniso.txt"):
        k = hs.index(h)
        ours = fabricated_errors[(case, scheme, k)]
        assert abs(ours / float(err) - 1.0) <= 0.06, (case, scheme, h, ours, err)
        if order != "-":
            o = np.log2(fabricated_errors[(case, scheme, k - 1)] / ours)
            assert abs(o - float(order)) <= 0.02, (case, scheme, h, o, order)


def test_rlm3_comparable_to_p1(fabricated_errors):
    for case in ("iso", "aniso"):
        for k in range(4):
            e3, e1, er = (fabricated_errors[(case, s, k)] for s in ("rlm3", "p1", "rlm"))
            assert e3 < 1.15 * e1 and e3 < 0.4 * er, (case, k, e3, e1, er)
        o = np.log2(fabricated_errors[(case, "rlm3", 2)] / fabricated_errors[(case, "rlm3", 3)])
        assert abs(o - 2.0) < 0.05


def _exact_problem(psi, dpsi, n=9, eps=0.7, ss=1.3, sa=0.4):
    """Slab with the exact solution psi(x, mu) (q from eq-1d with the discrete angular average)."""
    mu, w = gauss_ordinates(8)
    st = ss / eps + eps * sa
    phi = lambda x: sum(wl * psi(x, m) for m, wl in zip(mu, w))
    q = lambda x, m: (m * dpsi(x, m) + st * psi(x, m) - ss / eps * phi(x)) / eps
    return Slab(0.0, 1.3, n, 8, ss, sa, eps, q, lambda m: psi(0.0, m), lambda m: psi(1.3, m))


@pytest.mark.parametrize("name,psi,dpsi,exact_for", [
    ("constant", lambda x, m: 2.5 + 0 * x + 0 * m, lambda x, m: 0 * x + 0 * m, ("p0", "p1", "lm", "rlm", "rlm3")),
    ("linear", lambda x, m: 1.0 + 0.8 * x + 0 * m, lambda x, m: 0.8 + 0 * x + 0 * m, ("p1", "lm", "rlm", "rlm3")),
    ("aniso-linear", lambda x, m: m * x + 0.3, lambda x, m: m + 0 * x, ("p1", "rlm", "rlm3")),
])
def test_exact_states(name, psi, dpsi, exact_for):
    s = _exact_problem(psi, dpsi)
    for scheme in ("p0", "p1", "lm", "rlm", "rlm3"):
        err = s.l1_error(s.solve(scheme), psi)
        if scheme in exact_for:
            assert err < 1e-12, (name, scheme, err)
        else:
            assert err > 1e-4, (name, scheme, err)

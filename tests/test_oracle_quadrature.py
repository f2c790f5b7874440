"""Pins for the angular quadrature tables (inputs shared by the oracle and the CUDA path).

eq-polyquad: (i) sum w = 1, (ii) sum w Omega = 0, (iii) sum w Omega (x) Omega = Id/3; positive weights; no
direction on an axis (the sweeps need a definite upwind side); central symmetry (Theorem lem-B11).
"""
import numpy as np
import pytest

from workloads.quadrature import level_symmetric_2d, quadrant_of


@pytest.mark.parametrize("N,count", [(4, 12), (8, 40), (12, 84), (16, 144)])
def test_moments(N, count):
    ox, oy, w = level_symmetric_2d(N)
    assert len(w) == count == N * (N + 2) // 2
    assert np.all(w > 0)
    assert abs(w.sum() - 1) < 1e-14
    assert abs((w * ox).sum()) < 1e-14 and abs((w * oy).sum()) < 1e-14
    T = np.array([[(w * ox * ox).sum(), (w * ox * oy).sum()], [(w * ox * oy).sum(), (w * oy * oy).sum()]])
    assert np.abs(T - np.eye(2) / 3).max() < 1e-14
    assert np.abs(ox).min() > 0.1 and np.abs(oy).min() > 0.1
    assert np.all(ox * ox + oy * oy < 1)


@pytest.mark.parametrize("N", [4, 8, 12, 16])
def test_central_symmetry_and_quadrants(N):
    ox, oy, w = level_symmetric_2d(N)
    q = quadrant_of(ox, oy)
    m = len(w) // 4
    assert np.all(q == np.repeat(np.arange(4), m))
    for l in range(len(w)):
        k = np.nonzero((np.abs(ox + ox[l]) < 1e-15) & (np.abs(oy + oy[l]) < 1e-15))[0]
        assert len(k) == 1 and abs(w[k[0]] - w[l]) < 1e-16


def test_half_range_current():
    # sum over Omega_x > 0 of w Omega_x -> 1/4 (the half-range current of the unit sphere)
    for N in (8, 12, 16):
        ox, oy, w = level_symmetric_2d(N)
        assert abs((w * ox * (ox > 0)).sum() - 0.25) < 0.006


def test_s8_weights_lewis_miller():
    # LQ_8 point weights (Lewis & Miller, Table 4-1), normalised to 1 per octant: 0.1209877, 0.0907407,
    # 0.0925926 -- the set the paper's footnote on level-symmetric quadratures points to.
    ox, oy, w = level_symmetric_2d(8)
    vals = sorted(set(np.round(w[:10] * 4, 7)))
    assert np.allclose(vals, [0.0907407, 0.0925926, 0.1209877], atol=2e-7)

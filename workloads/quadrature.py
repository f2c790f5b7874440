"""Level-symmetric S_N angular quadrature projected to the unit disk (the 2D setting of eq-main).

Section 2.1 asks for positive weights with (i) sum w = 1, (ii) sum w Omega = 0 and (iii) sum w Omega (x) Omega
= Id / 3 (eq-polyquad); its footnote points to level-symmetric sets (Lewis & Miller).  The paper prints no
values, so the table is generated here from the standard LQ_N construction:

* level cosines ``mu_i^2 = mu_1^2 + (i - 1) * 2 (1 - 3 mu_1^2) / (N - 2)``, ``i = 1..N/2``;
* octant points ``(mu_i, mu_j, mu_k)`` with ``i + j + k = N/2 + 2`` (all lie on the unit sphere);
* one weight per permutation class, fixed by exact integration of the even monomials
  ``mu_x^{2a} mu_y^{2b} mu_z^{2c}`` of total degree <= N - 2 over the sphere;
* the 2D set keeps the upper hemisphere (``mu_z > 0``), projects to ``(Omega_x, Omega_y)`` and doubles the
  weights, giving ``n_Omega = N (N + 2) / 2`` directions (S4: 12, S8: 40, S12: 84, S16: 144).

Permutation symmetry makes (iii) exact for any class weights, and central symmetry makes (ii) exact, so the
degree-2 conditions hold to rounding whatever the higher-moment fit gives.  No direction has a zero
component.

Directions are returned grouped by quadrant in the order (+,+), (-,+), (-,-), (+,-), each quadrant holding
the same |Omega| pattern, so quadrant ``q`` occupies ``[q * n_Omega / 4, (q + 1) * n_Omega / 4)``.
"""
import numpy as np

# First level cosine of the standard LQ_N sets (Lewis & Miller, Table 4-1).
_MU1 = {2: 0.5773503, 4: 0.3500212, 6: 0.2666355, 8: 0.2182179, 10: 0.1893213, 12: 0.1672126,
        14: 0.1519859, 16: 0.1389568}


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def _octant(N):
    mu1 = _MU1[N]
    if N == 2:
        mu = np.array([mu1])
    else:
        d = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2)
        mu = np.sqrt(mu1 * mu1 + np.arange(N // 2) * d)
    pts = [(i, j, k) for i in range(N // 2) for j in range(N // 2) for k in range(N // 2)
           if i + j + k == N // 2 - 1]
    classes = sorted({tuple(sorted(p)) for p in pts})
    cid = [classes.index(tuple(sorted(p))) for p in pts]
    rows, rhs = [], []
    maxdeg = max(N - 2, 0)
    for a in range(maxdeg // 2 + 1):
        for b in range(a + 1):
            for c in range(b + 1):
                if 2 * (a + b + c) > maxdeg:
                    continue
                r = np.zeros(len(classes))
                for p, ci in zip(pts, cid):
                    r[ci] += mu[p[0]] ** (2 * a) * mu[p[1]] ** (2 * b) * mu[p[2]] ** (2 * c)
                rows.append(r)
                rhs.append(_dfact(2 * a - 1) * _dfact(2 * b - 1) * _dfact(2 * c - 1)
                           / _dfact(2 * (a + b + c) + 1))
    wc, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    wc = wc / sum(wc[ci] for ci in cid)          # octant weights sum to 1
    if np.any(wc <= 0):
        raise ValueError(f"LQ_{N} produced a non-positive weight")
    dirs = np.array([[mu[p[0]], mu[p[1]], mu[p[2]]] for p in pts])
    w = np.array([wc[ci] for ci in cid])
    return dirs, w


def level_symmetric_2d(N):
    """Return ``(ox, oy, w)`` (float64 arrays of length N(N+2)/2) for the 2D-projected LQ_N set."""
    if N not in _MU1:
        raise ValueError(f"unsupported S_N order {N}")
    dirs, w = _octant(N)
    # octant weights sum to 1; 8 octants -> divide by 8; keep the 4 upper octants and double.
    w2 = w / 4.0
    signs = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    ox, oy, ww = [], [], []
    for sx, sy in signs:
        ox.append(sx * dirs[:, 0])
        oy.append(sy * dirs[:, 1])
        ww.append(w2)
    return np.concatenate(ox), np.concatenate(oy), np.concatenate(ww)


def quadrant_of(ox, oy):
    """Quadrant index in the order (+,+)=0, (-,+)=1, (-,-)=2, (+,-)=3."""
    ox = np.asarray(ox)
    oy = np.asarray(oy)
    return np.where(oy > 0, np.where(ox > 0, 0, 1), np.where(ox < 0, 2, 3))

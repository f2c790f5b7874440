"""Seeded random problems shared by the tests (inputs only)."""
import numpy as np

from workloads.problems import uniform_problem


def random_problem(n, N, eps, seed, alpha=True, q_per_angle=True, sig=(0.2, 3.0), siga=(0.1, 2.0), ny=0):
    """n x ny cells (ny = 0: square) with seeded random per-cell cross sections, source and inflow data."""
    rng = np.random.default_rng(seed)
    p = uniform_problem(n, N, 1.0, 1.0, 1.0, eps=eps, name=f"rand-{n}x{ny or n}-S{N}-eps{eps:g}-{seed}", ny=ny)
    p.sigma_s = rng.uniform(*sig, p.nx)
    p.sigma_a = rng.uniform(*siga, p.nx)
    p.q = rng.uniform(0.0, 2.0, (p.nang, p.nx, 4) if q_per_angle else (p.nx, 4))
    if alpha:
        p.alpha = rng.uniform(0.0, 1.0, (p.nang, 4, max(n, p.rows), 2))
    return p


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

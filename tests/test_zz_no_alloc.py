"""The allocation-free operator application, lmdg_sweep_noalloc, against lmdg_sweep.

Some callers cannot call cudaMalloc (a framework that owns all device memory through its own pool, a loop
that cannot take cudaMalloc's implicit synchronisation, an embedding runtime that only hands over buffers);
lmdg_sweep_noalloc serves them from a fixed device scratch array.  This file is collected last so that a run
stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

from tests.helpers import random_problem, rel

pytestmark = pytest.mark.gpu


def _fn():
    from paper_1907_01027_gb300 import lmdg
    L = lmdg._lib()
    f = L.lmdg_sweep_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp,
                  ctypes.c_longlong, vp]
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("variant,code", [("std", 0), ("lm", 1), ("rlm", 2)])
def test_noalloc_matches_context_sweep_twice(variant, code):
    import torch
    from paper_1907_01027_gb300 import Context
    f = _fn()
    p = random_problem(70, 8, 0.5, 81, alpha=False, q_per_angle=False)
    ctx = Context(p, variant)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    ox, oy, w = dev(p.ox), dev(p.oy), dev(p.w)
    sigt = dev(p.sigma_s / p.eps + p.eps * p.sigma_a)
    sse = dev(p.sigma_s / p.eps)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(82)
    for call in range(2):
        x = rng.standard_normal((p.nx, 4))
        ref = ctx.sweep(x)
        xd = dev(x)
        yd = torch.full_like(xd, float("nan"))
        rc = f(code, p.n, p.h, p.nang, ox.data_ptr(), oy.data_ptr(), w.data_ptr(), sigt.data_ptr(), sse.data_ptr(),
               xd.data_ptr(), yd.data_ptr(), 1 << 26, stream)
        assert rc == 0, (call, rc)
        assert rel(yd.cpu().numpy(), ref) < 1e-12, call
    ctx.close()


def _many_directions(n_omega):
    """A valid quadrature with n_omega directions (n_omega / 4 per quadrant, |Omega| = 0.9, equal weights)."""
    m = n_omega // 4
    th = (np.arange(m) + 0.5) * (0.5 * np.pi / m)
    a, b = 0.9 * np.cos(th), 0.9 * np.sin(th)
    ox = np.concatenate([a, -a, -a, a])
    oy = np.concatenate([b, b, -b, -b])
    return ox, oy, np.full(n_omega, 1.0 / n_omega)


@pytest.mark.parametrize("variant,code", [("std", 0), ("lm", 1), ("rlm", 2)])
@pytest.mark.parametrize("n_omega", [40, 144, 1024])
def test_noalloc_launch_shapes(variant, code, n_omega):
    """The fixed launch shape of the allocation-free path grows with the direction count (one group of up to
    8 warps x 2 directions at 40, 3 directions per warp at 144, 8 groups of 8 warps x 4 at 1024): each against
    lmdg_sweep on a 16 x 16 mesh."""
    import torch
    from paper_1907_01027_gb300 import Context
    f = _fn()
    p = random_problem(16, 8, 0.7, 83, alpha=False, q_per_angle=False)
    if n_omega == 144:
        p = random_problem(16, 16, 0.7, 83, alpha=False, q_per_angle=False)
    elif n_omega == 1024:
        p.ox, p.oy, p.w = _many_directions(n_omega)
    assert p.nang == n_omega
    ctx = Context(p, variant)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    ox, oy, w = dev(p.ox), dev(p.oy), dev(p.w)
    sigt = dev(p.sigma_s / p.eps + p.eps * p.sigma_a)
    sse = dev(p.sigma_s / p.eps)
    stream = torch.cuda.current_stream().cuda_stream
    x = np.random.default_rng(84).standard_normal((p.nx, 4))
    ref = ctx.sweep(x)
    xd = dev(x)
    yd = torch.full_like(xd, float("nan"))
    rc = f(code, p.n, p.h, p.nang, ox.data_ptr(), oy.data_ptr(), w.data_ptr(), sigt.data_ptr(), sse.data_ptr(),
           xd.data_ptr(), yd.data_ptr(), 1 << 26, stream)
    assert rc == 0
    assert rel(yd.cpu().numpy(), ref) < 1e-12
    ctx.close()


def test_noalloc_rejects_unsorted_directions():
    """Directions not grouped by quadrant (here the level-symmetric set sorted by Omega_y, which interleaves the
    quadrants) are refused with LMDG_ERR_QUAD instead of giving a wrong result."""
    import torch
    f = _fn()
    p = random_problem(16, 8, 0.7, 85, alpha=False, q_per_angle=False)
    order = np.argsort(p.oy, kind="stable")          # mixes the quadrants
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    ox, oy, w = dev(p.ox[order]), dev(p.oy[order]), dev(p.w[order])
    sigt = dev(p.sigma_s / p.eps + p.eps * p.sigma_a)
    sse = dev(p.sigma_s / p.eps)
    xd = dev(np.ones((p.nx, 4)))
    yd = torch.empty_like(xd)
    rc = f(0, p.n, p.h, p.nang, ox.data_ptr(), oy.data_ptr(), w.data_ptr(), sigt.data_ptr(), sse.data_ptr(),
           xd.data_ptr(), yd.data_ptr(), 1 << 26, torch.cuda.current_stream().cuda_stream)
    assert rc == -2


def test_noalloc_rejects_oversized_problem():
    import torch
    f = _fn()
    n = 1024
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = f(0, n, 1.0 / n, 144, d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(),
           d.data_ptr(), 1 << 26, None)
    assert rc == -1

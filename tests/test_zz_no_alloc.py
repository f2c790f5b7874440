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


def test_noalloc_rejects_oversized_problem():
    import torch
    f = _fn()
    n = 1024
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = f(0, n, 1.0 / n, 144, d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(),
           d.data_ptr(), 1 << 26, None)
    assert rc == -1

"""Argument validation of lmdg_setup (host logic, runs before any device work, so it is checked on the CPU)."""
import ctypes

import numpy as np
import pytest

from workloads.problems import uniform_problem


@pytest.fixture(scope="module")
def L():
    from paper_1907_01027_gb300 import lmdg
    try:
        return lmdg._lib()
    except ImportError:
        pytest.skip("liblmdg not built")


def _setup(L, p, eps=None, variant=0, ox=None, oy=None, w=None, nang=None):
    from paper_1907_01027_gb300.lmdg import Mesh, Quad
    ox = np.ascontiguousarray(p.ox if ox is None else ox)
    oy = np.ascontiguousarray(p.oy if oy is None else oy)
    w = np.ascontiguousarray(p.w if w is None else w)
    mesh = Mesh(p.n, p.rows, p.x0, p.y0, p.h)
    quad = Quad(len(w) if nang is None else nang, ox.ctypes.data, oy.ctypes.data, w.ctypes.data)
    ss = np.ascontiguousarray(p.sigma_s)
    sa = np.ascontiguousarray(p.sigma_a)
    q = np.ascontiguousarray(p.q)
    h = ctypes.c_void_p()
    rc = L.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), ss.ctypes.data, sa.ctypes.data,
                      q.ctypes.data, 1, None, 1, float(p.eps if eps is None else eps), variant, None)
    if rc == 0:
        L.lmdg_destroy(h)
    return rc


def test_invalid_arguments_rejected(L):
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    assert _setup(L, p, eps=0.0) == -1
    assert _setup(L, p, eps=-1.0) == -1
    assert _setup(L, p, variant=4) == -1
    assert _setup(L, p, variant=-1) == -1
    bad = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    bad.sigma_a[3] = -0.1
    assert _setup(L, bad) == -1
    zero = uniform_problem(4, 4, 0.0, 0.0, 1.0)             # sigma_t = 0
    assert _setup(L, zero) == -1


def test_invalid_quadrature_rejected(L):
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    ox = p.ox.copy()
    ox[0] = 0.0                                                # a direction on an axis
    assert _setup(L, p, ox=ox) == -2
    w = p.w * 1.01                                             # weights not summing to 1
    assert _setup(L, p, w=w) == -2
    assert _setup(L, p, nang=len(p.w) - 1) == -2               # not a multiple of 4
    oy = p.oy.copy()
    oy[0] = -oy[0]                                             # unequal quadrant populations
    assert _setup(L, p, oy=oy) == -2


def test_valid_arguments_reach_the_device(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("valid setup is exercised by the GPU tests")
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    assert _setup(L, p) == -4                                  # validated, then no CUDA device here


def test_suppress_option_validated(L):
    """The suppression switch is RLMDG's only and takes 0 or 1."""
    from paper_1907_01027_gb300.lmdg import Mesh, Quad, Options
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    mesh = Mesh(p.n, p.rows, p.x0, p.y0, p.h)
    arrs = [np.ascontiguousarray(a) for a in (p.ox, p.oy, p.w, p.sigma_s, p.sigma_a, p.q)]
    quad = Quad(len(p.w), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data)
    for variant, flag in ((0, 1), (1, 1), (2, 2), (2, -1)):
        o = Options()
        L.lmdg_default_options(ctypes.byref(o))
        o.suppress = flag
        h = ctypes.c_void_p()
        rc = L.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), arrs[3].ctypes.data,
                          arrs[4].ctypes.data, arrs[5].ctypes.data, 1, None, 1, 1.0, variant, ctypes.byref(o))
        assert rc == -1, (variant, flag)


def test_recon_option_validated(L):
    """The reconstructions (1: three-cell RLMDG*, 2: Q1-type) are RLMDG's only, take 0, 1 or 2 and exclude
    suppression."""
    from paper_1907_01027_gb300.lmdg import Mesh, Quad, Options
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    mesh = Mesh(p.n, p.rows, p.x0, p.y0, p.h)
    arrs = [np.ascontiguousarray(a) for a in (p.ox, p.oy, p.w, p.sigma_s, p.sigma_a, p.q)]
    quad = Quad(len(p.w), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data)
    for variant, recon, supp in ((0, 1, 0), (1, 1, 0), (3, 1, 0), (2, 3, 0), (2, -1, 0), (2, 1, 1), (2, 2, 1),
                                 (0, 2, 0), (1, 2, 0)):
        o = Options()
        L.lmdg_default_options(ctypes.byref(o))
        o.recon = recon
        o.suppress = supp
        h = ctypes.c_void_p()
        rc = L.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), arrs[3].ctypes.data,
                          arrs[4].ctypes.data, arrs[5].ctypes.data, 1, None, 1, 1.0, variant, ctypes.byref(o))
        assert rc == -1, (variant, recon, supp)


def test_resid_option_validated(L):
    """The residual arithmetic takes LMDG_RESID_FP64 (0) or LMDG_RESID_F32X2 (1) only."""
    from paper_1907_01027_gb300.lmdg import Mesh, Quad, Options
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    mesh = Mesh(p.n, p.rows, p.x0, p.y0, p.h)
    arrs = [np.ascontiguousarray(a) for a in (p.ox, p.oy, p.w, p.sigma_s, p.sigma_a, p.q)]
    quad = Quad(len(p.w), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data)
    for resid in (-1, 2, 7):
        o = Options()
        L.lmdg_default_options(ctypes.byref(o))
        assert o.resid == 0
        o.resid = resid
        h = ctypes.c_void_p()
        rc = L.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), arrs[3].ctypes.data,
                          arrs[4].ctypes.data, arrs[5].ctypes.data, 1, None, 1, 1.0, 0, ctypes.byref(o))
        assert rc == -1, resid


def test_precond_option_validated(L):
    """The preconditioner takes 0, 1, 2 (the vertex diffusion correction) or 3 (with the cell-block step), and 2
    and 3 are refused for P0-DG, whose scheme has no diffusion limit."""
    from paper_1907_01027_gb300.lmdg import Mesh, Quad, Options
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    mesh = Mesh(p.n, p.rows, p.x0, p.y0, p.h)
    arrs = [np.ascontiguousarray(a) for a in (p.ox, p.oy, p.w, p.sigma_s, p.sigma_a, p.q)]
    quad = Quad(len(p.w), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data)
    for variant, pc in ((0, -1), (1, 4), (3, 2), (3, 3)):
        o = Options()
        L.lmdg_default_options(ctypes.byref(o))
        assert o.precond == 1
        o.precond = pc
        h = ctypes.c_void_p()
        rc = L.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), arrs[3].ctypes.data,
                          arrs[4].ctypes.data, arrs[5].ctypes.data, 1, None, 1, 1.0, variant, ctypes.byref(o))
        assert rc == -1, (variant, pc)


def test_mesh_and_alpha_layout_validated(L):
    """Meshes need at least one cell along each axis; the inflow data layout is 0 (one value) or 1 (per face)."""
    from paper_1907_01027_gb300.lmdg import Mesh, Quad
    p = uniform_problem(4, 4, 1.0, 1.0, 1.0)
    arrs = [np.ascontiguousarray(a) for a in (p.ox, p.oy, p.w, p.sigma_s, p.sigma_a, p.q)]
    quad = Quad(len(p.w), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data)
    alpha = np.zeros(4 * 4 * len(p.w) * 2)
    for (nx, ny), lay, a in (((0, 4), 1, None), ((4, 0), 1, None), ((4, 4), 2, alpha), ((4, 4), -1, alpha)):
        mesh = Mesh(nx, ny, p.x0, p.y0, p.h)
        h = ctypes.c_void_p()
        rc = L.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), arrs[3].ctypes.data,
                          arrs[4].ctypes.data, arrs[5].ctypes.data, 1, None if a is None else a.ctypes.data, lay,
                          1.0, 0, None)
        assert rc == -1, (nx, ny, lay)


def test_shard_entry_points_reject_bad_arguments(L):
    """The angle-sharding calls check their arguments on the host before any device work: a missing context or
    buffer, a shard outside [0, nshards), nshards outside [1, 4096], host pointers, and float-float with FP32."""
    import ctypes as ct
    sets, chunk = ct.c_int(0), ct.c_int(0)
    nbytes = ct.c_size_t(0)
    assert L.lmdg_shard_layout(None, 0, 2, ct.byref(sets), ct.byref(chunk), ct.byref(nbytes)) == -1
    buf = (ct.c_double * 8)()
    assert L.lmdg_sweep_shard(None, buf, buf, 0, 2, 0, None) == -1
    assert L.lmdg_sweep_combine(None, buf, buf, buf, 0, None) == -1
    fake = ct.c_void_p(1)   # never dereferenced: each call below fails its checks before it touches the context
    assert L.lmdg_shard_layout(fake, 0, 0, None, None, None) == -1
    assert L.lmdg_shard_layout(fake, 0, 4097, None, None, None) == -1
    assert L.lmdg_shard_layout(fake, 2 | 16, 2, None, None, None) == -1       # FP32 and float-float
    assert L.lmdg_sweep_shard(fake, buf, buf, 2, 2, 0, None) == -1            # shard >= nshards
    assert L.lmdg_sweep_shard(fake, buf, buf, -1, 2, 0, None) == -1
    assert L.lmdg_sweep_shard(fake, buf, None, 0, 2, 0, None) == -1           # no partial buffer
    assert L.lmdg_sweep_shard(fake, buf, buf, 0, 2, 8, None) == -1            # host pointers
    assert L.lmdg_sweep_shard(fake, buf, buf, 0, 2, 16 | 4, None) == -1       # float-float storing
    assert L.lmdg_sweep_combine(fake, buf, buf, buf, 4, None) == -1           # storing flag
    assert L.lmdg_sweep_combine(fake, buf, buf, buf, 2 | 16, None) == -1

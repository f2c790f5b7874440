"""ctypes binding of liblmdg with the same entry points as ``include/lmdg.h`` (argument marshalling only).

Vectors may be numpy arrays (host; the call sets LMDG_HOST_PTRS) or torch CUDA tensors (device pointers on the
current torch stream).  Every compute step runs in the library's kernels.
"""
import ctypes
import os

import numpy as np

from . import buildlib as _build_mod

STD, LM, RLM, P0 = 0, 1, 2, 3
VARIANTS = {"std": STD, "lm": LM, "rlm": RLM, "p0": P0}
FP64, FP32, FP32_BF16STORE = 0, 1, 2
SWEEP_SOURCE, SWEEP_FP32, SWEEP_STORE, HOST_PTRS, SWEEP_F32X2, SOLVE_EXACT_REF = 1, 2, 4, 8, 16, 32
RESID_FP64, RESID_F32X2 = 0, 1
ERR_TIMEOUT, ERR_NOTCONV, ERR_BREAKDOWN, ERR_STATE = -6, -5, -7, -8


class LmdgError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {_lib().lmdg_strerror(code).decode()} ({code})")


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("h", ctypes.c_double)]


class Quad(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("ox", ctypes.c_void_p), ("oy", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("precond", ctypes.c_int), ("spin_limit", ctypes.c_longlong), ("device", ctypes.c_int),
                ("suppress", ctypes.c_int), ("recon", ctypes.c_int), ("resid", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("sweeps_fp64", ctypes.c_int),
                ("sweeps_fp32", ctypes.c_int), ("resid0", ctypes.c_double), ("resid", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("sweep_ms_fp64", ctypes.c_double),
                ("sweep_ms_fp32", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("sweeps_f32x2", ctypes.c_int), ("sweep_ms_f32x2", ctypes.c_double), ("kappa_est", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def build(force=False):
    return _build_mod.build(force=force)


def _lib():
    global _LIB
    if _LIB is None:
        path = os.environ.get("LMDG_LIB") or _build_mod.LIB
        if not os.path.exists(path):
            raise ImportError(f"liblmdg is not built ({path}); run paper_1907_01027_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "lmdg_default_options": ([vp], ip),
            "lmdg_strerror": ([ip], ctypes.c_char_p),
            "lmdg_setup": ([vp, vp, vp, vp, vp, vp, ip, vp, ip, dp, ip, vp], ip),
            "lmdg_sweep": ([vp, vp, vp, ip, vp], ip),
            "lmdg_solve": ([vp, vp, vp, vp, vp, ip, vp], ip),
            "lmdg_get_psi": ([vp, vp, ip, vp], ip),
            "lmdg_adjoint": ([vp, vp, vp, vp, vp, vp, vp, ip, vp], ip),
            "lmdg_b11_apply": ([vp, vp, vp, ip, vp], ip),
            "lmdg_b11_solve": ([vp, vp, vp, dp, vp, ip, vp], ip),
            "lmdg_precond_apply": ([vp, vp, vp, ip, vp], ip),
            "lmdg_info": ([vp, vp, vp, vp, vp], ip),
            "lmdg_shard_layout": ([vp, ip, ip, vp, vp, vp], ip),
            "lmdg_sweep_shard": ([vp, vp, vp, ip, ip, ip, vp], ip),
            "lmdg_sweep_combine": ([vp, vp, vp, vp, ip, vp], ip),
            "lmdg_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def default_options(**kw):
    o = Options()
    _lib().lmdg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    """(pointer, is_host) of a numpy array or a torch tensor."""
    if a is None:
        return None, True
    if isinstance(a, np.ndarray):
        return a.ctypes.data, True
    return a.data_ptr(), not a.is_cuda


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def pack_alpha(alpha, ncol, nrow):
    """Inflow data [n_Omega][4][max(ncol, nrow)][2] (sides west, east: nrow faces; south, north: ncol faces, each
    in its first entries) to the library's face list [n_Omega][2 nrow + 2 ncol][2]."""
    a = np.asarray(alpha, dtype=np.float64)
    return np.ascontiguousarray(np.concatenate([a[:, 0, :nrow], a[:, 1, :nrow], a[:, 2, :ncol], a[:, 3, :ncol]],
                                               axis=1))


class Context:
    """One problem on one GPU (lmdg_setup ... lmdg_destroy).  The problem's mesh has ``n`` cells along x and
    ``rows`` along y; a scalar ``alpha`` is the same inflow value on every face and direction."""

    def __init__(self, problem, variant, **opts):
        self.lib = _lib()
        p = problem
        self.n, self.nx, self.nang = p.n, p.nx, p.nang
        self.rows = getattr(p, "rows", p.n)
        self.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (p.ox, p.oy, p.w)]
        mesh = Mesh(p.n, self.rows, p.x0, p.y0, p.h)
        quad = Quad(p.nang, *[a.ctypes.data for a in self._keep])
        ss = np.ascontiguousarray(p.sigma_s, dtype=np.float64)
        sa = np.ascontiguousarray(p.sigma_a, dtype=np.float64)
        q = np.ascontiguousarray(p.q, dtype=np.float64)
        q_layout = 2 if q.ndim == 3 else 1
        if p.alpha is None:
            al, al_layout = None, 1
        elif np.ndim(p.alpha) == 0:
            al, al_layout = np.array([float(p.alpha)]), 0
        else:
            al, al_layout = pack_alpha(p.alpha, p.n, self.rows), 1
        self.options = default_options(**opts)
        h = ctypes.c_void_p()
        rc = self.lib.lmdg_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), ss.ctypes.data,
                                 sa.ctypes.data, q.ctypes.data, q_layout, None if al is None else al.ctypes.data,
                                 al_layout, float(p.eps), self.variant, ctypes.byref(self.options))
        if rc:
            raise LmdgError(rc, "lmdg_setup")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lmdg_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, rc, what, allow=()):
        if rc and rc not in allow:
            raise LmdgError(rc, what)
        return rc

    def sweep(self, x, y=None, flags=0):
        """lmdg_sweep: y = K x (or K x - b with SWEEP_SOURCE).  numpy in -> numpy out (host pointers)."""
        xp, host = _ptr(x)
        if host:
            x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.nx, 4)
            y = np.empty_like(x) if y is None else y
            rc = self.lib.lmdg_sweep(self.h, x.ctypes.data, y.ctypes.data, flags | HOST_PTRS, None)
        else:
            import torch
            y = torch.empty_like(x) if y is None else y
            rc = self.lib.lmdg_sweep(self.h, xp, y.data_ptr(), flags, _stream())
        self._check(rc, "lmdg_sweep")
        return y

    def solve(self, x0=None, want_x=True, want_phi=True, device=False, allow_stall=False, exact_ref=False,
              phi_out=None):
        """lmdg_solve.  Returns (x, phi, stats dict, status).  LMDG_ERR_NOTCONV returns normally (outputs written);
        with ``allow_stall`` so does LMDG_ERR_BREAKDOWN from a residual that stopped decreasing (a solve driven
        below what the arithmetic can reach).  ``exact_ref``: LMDG_SOLVE_EXACT_REF.  ``phi_out``: a host array
        [N][4] of float64 (pinned memory, for instance) that receives phi instead of a new one."""
        st = Stats()
        fl = SOLVE_EXACT_REF if exact_ref else 0
        if device:
            import torch
            x = torch.empty((self.nx, 4), dtype=torch.float64, device="cuda") if want_x else None
            phi = torch.empty((self.nx, 4), dtype=torch.float64, device="cuda") if want_phi else None
            rc = self.lib.lmdg_solve(self.h, None if x0 is None else x0.data_ptr(),
                                     None if x is None else x.data_ptr(), None if phi is None else phi.data_ptr(),
                                     ctypes.byref(st), fl, _stream())
        else:
            x = np.empty((self.nx, 4)) if want_x else None
            if phi_out is not None:
                if phi_out.dtype != np.float64 or phi_out.shape != (self.nx, 4) or not phi_out.flags.c_contiguous:
                    raise ValueError("phi_out must be a C-contiguous float64 array of shape (N, 4)")
                phi = phi_out
            else:
                phi = np.empty((self.nx, 4)) if want_phi else None
            x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
            rc = self.lib.lmdg_solve(self.h, None if x0a is None else x0a.ctypes.data,
                                     None if x is None else x.ctypes.data, None if phi is None else phi.ctypes.data,
                                     ctypes.byref(st), HOST_PTRS | fl, None)
        self._check(rc, "lmdg_solve", allow=(ERR_NOTCONV, ERR_BREAKDOWN) if allow_stall else (ERR_NOTCONV,))
        return x, phi, st.as_dict(), rc

    # ---- angle sharding (lmdg_shard_layout, lmdg_sweep_shard, lmdg_sweep_combine)
    def shard_layout(self, nshards, flags=0):
        """(sets, sets per chunk, bytes per chunk) of the partial sets for the arithmetic of ``flags``."""
        sets, chunk = ctypes.c_int(0), ctypes.c_int(0)
        nbytes = ctypes.c_size_t(0)
        self._check(self.lib.lmdg_shard_layout(self.h, flags, nshards, ctypes.byref(sets), ctypes.byref(chunk),
                                               ctypes.byref(nbytes)), "lmdg_shard_layout")
        return sets.value, chunk.value, nbytes.value

    def sweep_shard(self, x, parts, shard, nshards, flags=0):
        """lmdg_sweep_shard on torch CUDA tensors: chunk ``shard`` of ``parts`` (nshards * chunk bytes)."""
        self._check(self.lib.lmdg_sweep_shard(self.h, x.data_ptr(), parts.data_ptr(), shard, nshards, flags,
                                              _stream()), "lmdg_sweep_shard")

    def sweep_combine(self, x, parts, y=None, flags=0):
        """lmdg_sweep_combine on torch CUDA tensors: y = K x (K x - b with SWEEP_SOURCE) from complete partials."""
        import torch
        y = torch.empty_like(x) if y is None else y
        self._check(self.lib.lmdg_sweep_combine(self.h, x.data_ptr(), parts.data_ptr(), y.data_ptr(), flags,
                                                _stream()), "lmdg_sweep_combine")
        return y

    def get_psi(self):
        per = 4 if self.variant == STD else 1
        out = np.empty((self.nang, self.nx, per) if per == 4 else (self.nang, self.nx))
        self._check(self.lib.lmdg_get_psi(self.h, out.ctypes.data, HOST_PTRS, None), "lmdg_get_psi")
        return out

    def b11_apply(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.nx, 3)
        y = np.empty_like(x)
        self._check(self.lib.lmdg_b11_apply(self.h, x.ctypes.data, y.ctypes.data, HOST_PTRS, None), "lmdg_b11_apply")
        return y

    def precond_apply(self, x):
        """lmdg_precond_apply: y = Minv x, the right preconditioner of lmdg_solve (host arrays)."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.nx, 4)
        y = np.empty_like(x)
        self._check(self.lib.lmdg_precond_apply(self.h, x.ctypes.data, y.ctypes.data, HOST_PTRS, None),
                    "lmdg_precond_apply")
        return y

    def b11_solve(self, r, tol=1e-14):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(self.nx, 3)
        z = np.empty_like(r)
        it = ctypes.c_int(0)
        self._check(self.lib.lmdg_b11_solve(self.h, r.ctypes.data, z.ctypes.data, tol, ctypes.byref(it), HOST_PTRS,
                                            None), "lmdg_b11_solve")
        return z, it.value

    def adjoint(self, g):
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = [np.empty(self.nx) for _ in range(3)]
        J = ctypes.c_double(0)
        st = Stats()
        self._check(self.lib.lmdg_adjoint(self.h, g.ctypes.data, out[0].ctypes.data, out[1].ctypes.data,
                                          out[2].ctypes.data, ctypes.byref(J), ctypes.byref(st), HOST_PTRS, None),
                    "lmdg_adjoint")
        return J.value, out[0], out[1], out[2], st.as_dict()

"""torch.autograd binding of the detector functional and its adjoint gradients (lmdg_solve / lmdg_adjoint).

J(sigma_s, sigma_a, q) = sum_K g_K int_K Psi_bar dx, with Psi the discrete solution of the standard or
low-memory scheme for per-cell cross sections and a per-cell constant source.  The forward pass runs
``lmdg_adjoint`` (the forward solve, the adjoint solve and the correlation sweep, all in the library's kernels)
and keeps the three per-cell gradients it returns; the backward pass scales them by the incoming gradient.
Argument marshalling only: no arithmetic of the method is done here.
"""
import copy

import numpy as np
import torch

from .lmdg import Context


class DetectorResponse(torch.autograd.Function):
    """``DetectorResponse.apply(sigma_s, sigma_a, q, problem, variant, g, options)`` -> J (0-d float64 tensor).

    sigma_s, sigma_a, q: [n*n] float64 tensors (any device; q is the per-cell constant source); problem: a
    ``workloads.Problem`` giving the mesh, quadrature, eps and inflow data (its own cross sections and source are
    replaced); variant: "std" or "lm"; g: [n*n] detector weights; options: dict of ``lmdg_options`` fields."""

    @staticmethod
    def forward(ctx, sigma_s, sigma_a, q, problem, variant, g, options=None):
        p = copy.copy(problem)
        p.sigma_s = sigma_s.detach().to("cpu", torch.float64).numpy().copy()
        p.sigma_a = sigma_a.detach().to("cpu", torch.float64).numpy().copy()
        qc = np.zeros((p.nx, 4))
        qc[:, 0] = q.detach().to("cpu", torch.float64).numpy()
        p.q = qc
        c = Context(p, variant, **(options or {}))
        try:
            J, dss, dsa, dq, _ = c.adjoint(np.asarray(g, dtype=np.float64))
        finally:
            c.close()
        dev = sigma_s.device
        ctx.save_for_backward(torch.from_numpy(dss).to(dev), torch.from_numpy(dsa).to(dev),
                              torch.from_numpy(dq).to(dev))
        return torch.tensor(J, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, grad_J):
        dss, dsa, dq = ctx.saved_tensors
        return grad_J * dss, grad_J * dsa, grad_J * dq, None, None, None, None


def detector_response(sigma_s, sigma_a, q, problem, variant, g, **options):
    """J = sum_K g_K int_K Psi_bar dx as a differentiable function of the per-cell sigma_s, sigma_a and q."""
    return DetectorResponse.apply(sigma_s, sigma_a, q, problem, variant, g, options)

"""The autograd binding of the detector functional (paper_1907_01027_gb300.autograd) on the GPU: gradients from
the adjoint (lmdg_adjoint) against torch.autograd.gradcheck's central differences of the forward functional, and
against the library call they wrap."""
import numpy as np
import pytest

from workloads.problems import config5

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["std", "lm"])
def test_gradcheck_detector_response(variant):
    import torch
    from paper_1907_01027_gb300.autograd import detector_response
    p = config5(n=6, N=4)
    g = p.info["detector"] + 0.25           # every cell in the functional, the detector cells more
    opts = dict(tol=1e-14, max_iters=20000)
    ss = torch.tensor(p.sigma_s, dtype=torch.float64, requires_grad=True)
    sa = torch.tensor(p.sigma_a, dtype=torch.float64, requires_grad=True)
    q = torch.tensor(p.q[:, 0], dtype=torch.float64, requires_grad=True)
    f = lambda a, b, c: detector_response(a, b, c, p, variant, g, **opts)
    # central differences with step 1e-6 on every input against the adjoint gradients
    assert torch.autograd.gradcheck(f, (ss, sa, q), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_backward_equals_library_adjoint():
    import torch
    from paper_1907_01027_gb300 import Context
    from paper_1907_01027_gb300.autograd import detector_response
    p = config5(n=16)
    g = p.info["detector"]
    ss = torch.tensor(p.sigma_s, dtype=torch.float64, requires_grad=True)
    sa = torch.tensor(p.sigma_a, dtype=torch.float64, requires_grad=True)
    q = torch.tensor(p.q[:, 0], dtype=torch.float64, requires_grad=True)
    J = detector_response(ss, sa, q, p, "std", g, tol=1e-13)
    (2.0 * J).backward()
    ctx = Context(p, "std", tol=1e-13)
    J0, dss, dsa, dq, _ = ctx.adjoint(g)
    ctx.close()
    assert float(J.detach()) == J0
    assert np.array_equal(ss.grad.numpy(), 2.0 * dss)
    assert np.array_equal(sa.grad.numpy(), 2.0 * dsa)
    assert np.array_equal(q.grad.numpy(), 2.0 * dq)

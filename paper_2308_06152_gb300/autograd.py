"""torch.autograd face of hz_gradient.

``misfit(m, desc, omega, src, rec_idx, d_obs)`` returns
J(m) = 1/2 sum_s ||S u_s - d_s||^2 for the squared slowness m (k^2 =
omega^2 m) as a differentiable scalar; its backward pass returns dJ/dm as
computed by the library's adjoint solve and imaging kernel (one forward and
one adjoint solve per shot, both on the GPU).
"""

import torch

from .api import Solver


class HelmholtzMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, desc, omega, src, rec_idx, d_obs, tol):
        m64 = m.detach().to(dtype=torch.float64)
        solver = Solver(desc, (omega * omega) * m64, device=m.device)
        J, grad, infos = solver.gradient(omega, src, rec_idx, d_obs, tol=tol)
        solver.close()
        ctx.save_for_backward(grad.to(dtype=m.dtype))
        ctx.infos = infos
        return torch.tensor(J, dtype=m.dtype, device=m.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ * grad, None, None, None, None, None, None


def misfit(m, desc, omega, src, rec_idx, d_obs, tol=1e-10):
    """Differentiable data misfit J(m); m: (ny, nx) CUDA tensor."""
    return HelmholtzMisfit.apply(m, desc, omega, src, rec_idx, d_obs, tol)

"""torch.autograd wrapper of the adjoint-state gradient (helmholtz_adjoint_grad).

``helmholtz_misfit(m, ...)`` returns J(m) = 1/2 sum_s || R Q_h v_s - d_s ||^2 for
the squared slowness m = 1/c^2 on every fine node (a CUDA float64 tensor of
shape (nz+1, ny+1, nx+1)); its backward pass returns dJ/dm computed by the
library (forward solves, adjoint solves with A_h^H, row-local derivatives of
A_h and Q_h; PML entries folded onto the physical node they copy).
"""
from __future__ import annotations

import torch

from . import Solver, default_params


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, grid, sources, receivers, d_obs):
        n, n_pml, h, omega, params, max_nrhs, gamma_max = grid
        c = torch.rsqrt(m.detach().to(torch.float64)).contiguous()
        s = Solver(n, n_pml, h, omega, c, params=params, max_nrhs=max_nrhs, gamma_max=gamma_max)
        try:
            J, g, stats = s.helmholtz_adjoint_grad(sources, receivers, d_obs)
        finally:
            s.close()
        ctx.save_for_backward(g)
        ctx.stats = stats
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g.to(grad_out.device), None, None, None, None


def helmholtz_misfit(m, n, n_pml, h, omega, sources, receivers, d_obs, params=None, max_nrhs=1,
                     gamma_max=1.119058):
    """Differentiable receiver misfit of the IOFD Helmholtz solution w.r.t. m = 1/c^2."""
    params = params or default_params()
    return _Misfit.apply(m, (n, n_pml, h, omega, params, max_nrhs, gamma_max), sources, receivers, d_obs)

"""torch.autograd.Function around the solve of D x = b.

Forward: x = D[U]^-1 b through the library's mixed-precision SAP-BiCGStab
solve (Algorithms 4 and 5 of arXiv:2109.10687).  Backward, for an upstream
gradient g = dL/dx (torch's convention for real losses of complex tensors,
so that dL = Re(g^dag dx)):

* grad_b = D^-dag g = gamma_5 D^-1 gamma_5 g          (the adjoint solve)
* grad_U = G with dL = sum Re tr(G^dag dU)             (hopping + clover
  leaf force from x and lambda = grad_b, the library's force kernel)

Both come from one call of qcd_grad.  Tensors are complex128 in the
canonical layout: b ``[t][z][y][x][3][4]``, U ``[t][z][y][x][4][3][3]``.
"""

import torch

from . import binding as B


class DiracSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, u, lattice, kappa, csw, params):
        lattice.set_gauge(u.detach())
        lattice.set_params(kappa, csw)
        lattice.build_clover()
        x, rc, info = lattice.solve(b.detach(), params=params)
        ctx.lattice = lattice
        ctx.params = params
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        lat = ctx.lattice
        eta = torch.view_as_real(grad_x.detach().to(torch.complex128).contiguous()).contiguous()
        xr = torch.view_as_real(x.contiguous()).contiguous()
        gb = torch.zeros_like(eta)
        gu = None
        if ctx.needs_input_grad[1]:
            lt, lz, ly, lx = lat.site_shape
            gu = torch.zeros((lt, lz, ly, lx, 4, 3, 3, 2), dtype=torch.float64, device=eta.device)
        B.qcd_grad(lat.ctx, eta, None, gb, gu, x=xr, lam=None, project=0, params=ctx.params)
        grad_b = torch.view_as_complex(gb) if ctx.needs_input_grad[0] else None
        grad_u = torch.view_as_complex(gu) if gu is not None else None
        return grad_b, grad_u, None, None, None, None


def solve(b, u, lattice, kappa, csw, params=None):
    """Differentiable x = D[U]^-1 b (see DiracSolve)."""
    if params is None:
        params = B.qcd_solve_params_default()
    return DiracSolve.apply(b, u, lattice, kappa, csw, params)

"""GPU gradients of L = Re(eta^dag D^-1 b) against the float64 oracle
gradient (hopping and clover parts, raw and su(3)-projected)."""

import numpy as np
import pytest
import torch

from gpu_util import Problem, rel_l2, to_np
from oracle import grad

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,domain,csw", [((4, 4, 4, 4), (2, 2, 2, 2), 1.0),
                                             ((8, 8, 8, 8), (4, 4, 4, 4), 1.0),
                                             ((4, 4, 4, 8), (2, 2, 2, 2), 0.0)])
def test_grad_matches_oracle(dims, domain, csw):
    from paper_2109_10687_gb300 import binding as B
    p = Problem(dims, domain, eps=0.3, kappa=0.12, csw=csw, seed=3000)
    try:
        eta, b = p.source(3001), p.source(3002)
        lam_ref, g_ref = grad.gradients(p.op, eta, b, tol=1e-13)
        pi_ref = grad.project_su3(g_ref, p.u)
        dev = p.lat.device
        e_t = torch.view_as_real(torch.from_numpy(eta).to(dev)).contiguous()
        b_t = torch.view_as_real(torch.from_numpy(b).to(dev)).contiguous()
        gb = torch.zeros_like(b_t)
        gu = torch.zeros(p.u.shape + (2,), dtype=torch.float64, device=dev)
        params = B.qcd_solve_params_default()
        params.tol = 1e-12
        B.qcd_grad(p.lat.ctx, e_t, b_t, gb, gu, project=0, params=params)
        assert rel_l2(to_np(torch.view_as_complex(gb)), lam_ref) < 1e-9
        assert rel_l2(to_np(torch.view_as_complex(gu)), g_ref) < 1e-5
        B.qcd_grad(p.lat.ctx, e_t, b_t, None, gu, project=1, params=params)
        assert rel_l2(to_np(torch.view_as_complex(gu)), pi_ref) < 1e-5
    finally:
        p.close()


def test_autograd_function_matches_oracle():
    """torch.autograd through the library solve: L = Re(eta^dag D^-1 b),
    gradients with respect to b and U against the float64 oracle."""
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.autograd import solve
    p = Problem((4, 4, 4, 8), (2, 2, 2, 2), eps=0.3, kappa=0.12, csw=1.0, seed=3100)
    try:
        eta, b = p.source(3101), p.source(3102)
        lam_ref, g_ref = grad.gradients(p.op, eta, b, tol=1e-13)
        dev = p.lat.device
        bt = torch.from_numpy(b).to(dev).requires_grad_(True)
        ut = torch.from_numpy(p.u).to(dev).requires_grad_(True)
        et = torch.from_numpy(eta).to(dev)
        params = B.qcd_solve_params_default()
        params.tol = 1e-12
        x = solve(bt, ut, p.lat, 0.12, 1.0, params)
        loss = torch.sum(torch.conj(et) * x).real
        loss.backward()
        x_ref = grad.solve_D(p.op, b)
        assert abs(loss.item() - np.vdot(eta.ravel(), x_ref.ravel()).real) < 1e-9 * abs(loss.item())
        assert rel_l2(to_np(bt.grad), lam_ref) < 1e-9
        assert rel_l2(to_np(ut.grad), g_ref) < 1e-5
    finally:
        p.close()

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

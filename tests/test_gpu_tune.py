"""The autotuners: SAP domain shapes by time to solution (qcd_tune_domain),
checked by solving with every shape it timed and recomputing the float64
true residual with the oracle."""

import numpy as np
import pytest
import torch

from gpu_util import to_np
from lattice_inputs import gaussian_spinor, random_su3_field
from oracle.dirac import CloverWilson
from oracle.gamma import gamma_chiral

pytestmark = pytest.mark.gpu


def test_domain_tuner_times_each_shape_and_each_solves():
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims, kappa, csw = (8, 8, 8, 8), 0.12, 1.0
    u = random_su3_field(dims, 0.3, 1001)
    b = gaussian_spinor(dims, 2001)
    ut = torch.view_as_real(torch.from_numpy(u)).cuda().contiguous()
    bt = torch.view_as_real(torch.from_numpy(b)).cuda().contiguous()
    p = B.qcd_solve_params_default()
    p.tol, p.inner_tol, p.sap_prec = 1e-10, 1e-5, B.PREC_HALF
    cands = [(4, 4, 4, 4), (2, 4, 4, 4), (4, 4, 2, 4), (2, 2, 2, 2), (8, 4, 4, 2), (3, 4, 4, 4)]
    best, secs = B.qcd_tune_domain(dims, ut, bt, kappa, csw, p, candidates=cands)
    # 8x4x4x2 needs L_x a multiple of 16 and 3 is not a power of two: skipped
    assert secs[(8, 4, 4, 2)] is None and secs[(3, 4, 4, 4)] is None
    timed = {c: t for c, t in secs.items() if t is not None}
    assert set(timed) == {(4, 4, 4, 4), (2, 4, 4, 4), (4, 4, 2, 4), (2, 2, 2, 2)}
    assert best == min(timed, key=timed.get)
    op = CloverWilson(u, kappa, csw, gamma_chiral(), bc_t=-1)
    for cand in timed:
        lat = Lattice(dims, cand, -1, "chiral").setup(u, kappa, csw)
        try:
            x, rc, info = lat.solve(b, tol=1e-10, inner_tol=1e-5, sap_prec="half")
            x = to_np(x)
            r = np.linalg.norm((b - op.D(x)).ravel()) / np.linalg.norm(b.ravel())
            assert rc == 0 and r < 1e-10, (cand, r)
        finally:
            lat.close()


def test_domain_tuner_default_list_and_no_candidate():
    from paper_2109_10687_gb300 import binding as B
    dims = (8, 8, 8, 8)
    u = torch.view_as_real(torch.from_numpy(random_su3_field(dims, 0.3, 1002))).cuda().contiguous()
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 2002))).cuda().contiguous()
    best, secs = B.qcd_tune_domain(dims, u, b, 0.12, 1.0)
    assert len(secs) == B.lib().qcd_tune_domain_default_count() and best in [(4, 4, 4, 4), (4, 4, 2, 4),
                                                                           (4, 4, 4, 2), (2, 2, 2, 2),
                                                                           (2, 4, 4, 8), (8, 4, 4, 2),
                                                                           (8, 8, 2, 2)]
    with pytest.raises(B.QcdError):
        B.qcd_tune_domain(dims, u, b, 0.12, 1.0, candidates=[(3, 3, 3, 3)])

"""Parity at the large workloads and at the degenerate cases of the method.

* 48^4 with 12 spin-colour point sources in one batched solve, in the launch
  configuration the benchmark times (float16-storage SAP, device-side graph
  loop, float64 defect correction): the residual b - D x of every right-hand
  side is recomputed by the site-by-site float64 oracle on sampled sites,
  around the source and at random, independently of the library's own D.
* kappa = 0, where the hopping term and the clover term (proportional to
  kappa) vanish and D = 1: the solve returns x = b.
* zero right-hand sides is rejected.
"""

import numpy as np
import pytest
import torch

from gpu_util import rel_l2, to_np
from lattice_inputs import gaussian_spinor, point_source, random_su3_field_fast
from oracle import pointwise
from oracle.gamma import gamma_chiral

pytestmark = pytest.mark.gpu


def _params(sap_prec="half", tol=1e-10, graph=2):
    from paper_2109_10687_gb300 import binding as B
    p = B.qcd_solve_params_default()
    p.tol, p.n_sap, p.n_jac, p.inner_tol, p.max_inner, p.use_graph = tol, 4, 4, 1e-5, 2000, graph
    p.sap_prec = {"half": B.PREC_HALF, "half_gauge": B.PREC_HALF_GAUGE, "single": B.PREC_SINGLE}[sap_prec]
    return p


def test_batched_point_sources_48x4_sampled():
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (48, 48, 48, 48)
    kappa, csw = 0.125, 1.1
    u = random_su3_field_fast(dims, 0.25, 1301)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(u, kappa, csw)
    try:
        srcs = np.stack([point_source(dims, c, s) for c in range(3) for s in range(4)])
        b = torch.view_as_real(torch.from_numpy(srcs)).cuda().contiguous()
        x = torch.zeros_like(b)
        rc, info = B.qcd_solve(lat.ctx, x, b, 12, _params())
        assert rc == 0 and info.true_resid < 1e-10
        xs = to_np(torch.view_as_complex(x))
        g = gamma_chiral()
        rng = np.random.default_rng(11)
        near = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 0, 0, 1), (47, 0, 0, 0), (0, 47, 0, 0), (0, 0, 0, 47)]
        for r in range(12):
            sites = near + [tuple(int(rng.integers(0, 48)) for _ in range(4)) for _ in range(4)]
            num = 0.0
            for c in sites:
                res = srcs[r][c[3], c[2], c[1], c[0]] - pointwise.D_at(u, xs[r], c, kappa, csw, g, -1)
                num += np.sum(np.abs(res) ** 2)
            # |b| = 1; the sampled residual is part of a global residual < 1e-10
            assert np.sqrt(num) < 1e-9, (r, np.sqrt(num))
    finally:
        lat.close()


def test_kappa_zero_gives_identity():
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (8, 8, 8, 8)
    u = random_su3_field_fast(dims, 0.3, 1011)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(u, 0.0, 1.0)
    try:
        b = gaussian_spinor(dims, 2011)
        for prec in ("half", "single"):
            x, rc, info = lat.solve(b, tol=1e-10, sap_prec=prec, inner_tol=1e-5)
            assert rc == 0 and info.true_resid < 1e-10
            assert rel_l2(to_np(x), b) < 1e-10   # D = 1: the residual is x - b itself
    finally:
        lat.close()


def test_zero_rhs_rejected():
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (8, 8, 8, 8)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(random_su3_field_fast(dims, 0.3, 1012), 0.12, 1.0)
    try:
        b = torch.zeros((1,) + lat.site_shape + (3, 4, 2), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        rc, _ = B.qcd_solve(lat.ctx, x, b, 0, _params(), raise_on_error=False)
        assert rc == B.QCD_ERR_ARG
    finally:
        lat.close()


def test_solve_64x4_sampled():
    """The 64^4 workload (eps 0.2, kappa 0.126, c_SW 1.1) at full size: the
    float32 D on 24 sampled sites and the mixed-precision solve's residual on
    48 sampled sites, both recomputed by the site-by-site float64 oracle."""
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (64, 64, 64, 64)
    kappa, csw = 0.126, 1.1
    u = random_su3_field_fast(dims, 0.2, 1501)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(u, kappa, csw)
    try:
        g = gamma_chiral()
        b = gaussian_spinor(dims, 2501)
        rng = np.random.default_rng(13)
        d32 = to_np(lat.apply_D(b, "single"))
        num = den = 0.0
        for _ in range(24):
            c = tuple(int(rng.integers(0, 64)) for _ in range(4))
            ref = pointwise.D_at(u, b, c, kappa, csw, g, -1)
            num += np.sum(np.abs(d32[c[3], c[2], c[1], c[0]] - ref) ** 2)
            den += np.sum(np.abs(ref) ** 2)
        assert np.sqrt(num / den) <= 1e-6
        del d32
        x, rc, info = lat.solve(b, tol=1e-10, inner_tol=1e-5, sap_prec="half", use_graph=2, max_inner=2000)
        assert rc == 0 and info.true_resid < 1e-10
        x = to_np(x)
        num = den = 0.0
        for _ in range(48):
            c = tuple(int(rng.integers(0, 64)) for _ in range(4))
            r = b[c[3], c[2], c[1], c[0]] - pointwise.D_at(u, x, c, kappa, csw, g, -1)
            num += np.sum(np.abs(r) ** 2)
            den += np.sum(np.abs(b[c[3], c[2], c[1], c[0]]) ** 2)
        assert np.sqrt(num / den) < 1e-8
    finally:
        lat.close()

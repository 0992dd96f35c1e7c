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


def test_ragged_batch_32_lattices_as_benchmarked():
    """The ragged batch the benchmark times (32 lattices with extents drawn
    from {8, 16}, kappa ~ U[0.115, 0.125], the same seeds), solved in shared
    launches: every lattice's residual b - D x recomputed by the site-by-site
    float64 oracle on 16 sampled sites, against 1e-9 of |b| there."""
    from lattice_inputs import random_su3_field
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    rng = np.random.default_rng(5000)
    lats, us, bs, kappas = [], [], [], []
    try:
        for i in range(32):
            dims = tuple(int(v) for v in rng.choice([8, 16], size=4))
            kappa = float(rng.uniform(0.115, 0.125))
            u = random_su3_field(dims, 0.3, 5000 + i)
            lats.append(Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(u, kappa, 1.0))
            us.append(u)
            kappas.append(kappa)
            bs.append(gaussian_spinor(dims, 7000 + i))
        bt = B.qcd_batch_create([l.ctx for l in lats])
        try:
            bd = [torch.view_as_real(torch.from_numpy(b)).cuda().contiguous() for b in bs]
            xd = [torch.zeros_like(b) for b in bd]
            rc, infos = B.qcd_batch_solve(bt, xd, bd, _params())
            assert rc == 0 and all(i.true_resid < 1e-10 for i in infos)
        finally:
            B.qcd_batch_destroy(bt)
        g = gamma_chiral()
        srng = np.random.default_rng(17)
        for i, (lat, u, b, x) in enumerate(zip(lats, us, bs, xd)):
            xn = to_np(torch.view_as_complex(x))
            num = den = 0.0
            for _ in range(16):
                c = tuple(int(srng.integers(0, lat.dims[mu])) for mu in range(4))
                r = b[c[3], c[2], c[1], c[0]] - pointwise.D_at(u, xn, c, kappas[i], 1.0, g, -1)
                num += np.sum(np.abs(r) ** 2)
                den += np.sum(np.abs(b[c[3], c[2], c[1], c[0]]) ** 2)
            assert np.sqrt(num / den) < 1e-9, (i, np.sqrt(num / den))
    finally:
        for l in lats:
            l.close()


@pytest.mark.parametrize("sap_prec,shape", [("half_gauge", 0), ("single", 1)])
def test_paper_domains_full_size(sap_prec, shape):
    """The paper-parameter workload of the benchmark line at full size:
    64x24x32x24 on the paper's 16x6x4x3 SAP domains (the cluster kernel with
    float16 links and C_inv; the one-CTA kernel in float32), n_sap 4, n_jac 2,
    solved to 1e-10; the residual recomputed by the site-by-site float64
    oracle on 48 sampled sites."""
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (64, 24, 32, 24)
    kappa, csw = 0.125, 1.0
    u = random_su3_field_fast(dims, 0.3, 1001)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(u, kappa, csw)
    try:
        B.qcd_set_sap_domain(lat.ctx, (16, 6, 4, 3))
        B.qcd_set_sap_shape(lat.ctx, shape)
        b = gaussian_spinor(dims, 2001)
        x, rc, info = lat.solve(b, tol=1e-10, inner_tol=1e-6 if sap_prec == "single" else 1e-5, n_sap=4, n_jac=2,
                                sap_prec=sap_prec, use_graph=2, max_inner=2000)
        assert rc == 0 and info.true_resid < 1e-10
        x = to_np(x)
        g = gamma_chiral()
        rng = np.random.default_rng(19)
        num = den = 0.0
        for _ in range(48):
            c = tuple(int(rng.integers(0, dims[mu])) for mu in range(4))
            r = b[c[3], c[2], c[1], c[0]] - pointwise.D_at(u, x, c, kappa, csw, g, -1)
            num += np.sum(np.abs(r) ** 2)
            den += np.sum(np.abs(b[c[3], c[2], c[1], c[0]]) ** 2)
        assert np.sqrt(num / den) < 1e-8
    finally:
        lat.close()


@pytest.mark.parametrize("sap_prec", ["half", "single"])
def test_one_launch_msap_at_32x4_equals_per_launch(sap_prec):
    """At the benchmark's 32^4 size (4096 domains, 2048 per colour), M_SAP in
    one launch (shape 3: every resident CTA in flight, items ordered by the
    neighbours' flags) equals the per-launch form (shape 0) bit for bit, for
    one and for two right-hand sides, twice in a row (the flags and counters
    are cleared between uses)."""
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (32, 32, 32, 32)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(random_su3_field_fast(dims, 0.3, 1001), 0.125, 1.0)
    try:
        prec = {"half": B.PREC_HALF, "single": B.PREC_SINGLE}[sap_prec]
        b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 2001))).cuda().contiguous()
        outs = {}
        for nrhs in (1, 2):
            a = lat.field("single", nrhs)
            src = b if nrhs == 1 else torch.stack([b, 0.5 * b.roll(1, 0)]).contiguous()
            B.qcd_import_spinor(lat.ctx, a, src, B.PREC_SINGLE, nrhs)
            for shape in (0, 3, 3):
                B.qcd_set_sap_shape(lat.ctx, shape)
                o = lat.field("single", nrhs)
                B.qcd_sap_apply_nrhs(lat.ctx, o, a, nrhs, 4, 4, prec, 0)
                outs.setdefault(nrhs, []).append(o.clone())
            assert B.qcd_device_status(lat.ctx) == B.QCD_OK
        for nrhs, (ref, *rest) in outs.items():
            for o in rest:
                assert torch.equal(o, ref), nrhs
    finally:
        B.qcd_set_sap_shape(lat.ctx, -1)
        lat.close()


def test_msap_32x4_twelve_rhs():
    """The benchmark's 32^4 lattice (4096 domains) with 12 right-hand sides
    through every SAP launch, float16 links and C_inv with float32 vectors:
    right-hand sides 0, 5 and 11 equal their single-rhs M_SAP bit for bit;
    M_SAP is linear to float32 rounding (M(b_0 + 2 b_1) against
    M b_0 + 2 M b_1); and A M_SAP stays close to the identity
    (|b - A M_SAP b| / |b| < 0.5), a property of the Schwarz preconditioner
    at any size."""
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    dims = (32, 32, 32, 32)
    lat = Lattice(dims, (4, 4, 4, 4), -1, "chiral").setup(random_su3_field_fast(dims, 0.3, 1001), 0.125, 1.0)
    try:
        b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 2201))).cuda()
        srcs = torch.stack([(1.0 + r / 12) * b.roll(r, r % 4) for r in range(12)]).contiguous()
        nb = B.qcd_field_bytes(lat.ctx, B.PREC_SINGLE, 1)
        a = lat.field("single", 12)
        B.qcd_import_spinor(lat.ctx, a, srcs, B.PREC_SINGLE, 12)
        o = lat.field("single", 12)
        B.qcd_sap_apply_nrhs(lat.ctx, o, a, 12, 4, 4, B.PREC_HALF_GAUGE, 0)
        one = lat.field("single", 1)
        for r in (0, 5, 11):
            B.qcd_sap_apply_nrhs(lat.ctx, one, a[r * nb:(r + 1) * nb], 1, 4, 4, B.PREC_HALF_GAUGE, 0)
            assert torch.equal(one, o[r * nb:(r + 1) * nb]), r
        m0 = lat.to_canonical(o[0:nb])
        m1 = lat.to_canonical(o[nb:2 * nb])
        comb = lat.to_internal(torch.view_as_complex(srcs[0] + 2.0 * srcs[1]))
        B.qcd_sap_apply_nrhs(lat.ctx, one, comb, 1, 4, 4, B.PREC_HALF_GAUGE, 0)
        lin = lat.to_canonical(one)
        assert rel_l2(to_np(lin), to_np(m0 + 2.0 * m1)) <= 1e-5
        B.qcd_sap_apply_nrhs(lat.ctx, o, a, 12, 4, 4, B.PREC_HALF_GAUGE, 1)
        for r in (0, 11):
            amb = to_np(lat.to_canonical(o[r * nb:(r + 1) * nb]))
            assert rel_l2(amb, to_np(torch.view_as_complex(srcs[r]))) < 0.5, r
        assert B.qcd_device_status(lat.ctx) == B.QCD_OK
    finally:
        lat.close()

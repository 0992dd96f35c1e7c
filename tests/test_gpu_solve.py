"""GPU solves of D x = b (Algorithms 4 and 5 with SAP) against the float64
oracle: true residual <= 1e-10 recomputed by the oracle, solution against the
oracle's own solve, the structure of Algorithm 5 against the oracle's literal
iterates, batched right-hand sides, failure statuses."""

import numpy as np
import pytest

from gpu_util import Problem, rel_l2, to_np
from lattice_inputs import gaussian_spinor, point_source
from oracle import solvers

pytestmark = pytest.mark.gpu


def true_resid(op, x, b):
    return float(np.linalg.norm((b - op.D(x)).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def c1():
    """8^4, eps 0.3, kappa 0.12, c_SW 1.0, 4^4 domains (the small solve workload)."""
    p = Problem((8, 8, 8, 8), (4, 4, 4, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1001)
    yield p
    p.close()


@pytest.fixture(scope="module")
def c1_ref(c1):
    b = gaussian_spinor(c1.dims, 2001)
    x, _, ok = solvers.bicgstab(c1.op.D, b, 1e-12, 3000)
    assert ok
    return b, x


@pytest.mark.parametrize("sap_prec", ["single", "half", "half_gauge"])
@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_solve_to_1e10(c1, c1_ref, sap_prec, use_graph):
    b, x_ref = c1_ref
    x, rc, info = c1.lat.solve(b, tol=1e-10, inner_tol=1e-6 if sap_prec == "single" else 1e-5,
                               n_sap=4, n_jac=4, sap_prec=sap_prec, use_graph=use_graph)
    x = to_np(x)
    assert rc == 0
    assert info.true_resid < 1e-10
    assert true_resid(c1.op, x, b) < 1e-10
    assert rel_l2(x, x_ref) < 1e-8
    assert 1 <= info.outer_iters <= 6


@pytest.mark.parametrize("residual_prec", [0, 1])
def test_solve_residual_precisions(c1, c1_ref, residual_prec):
    """Algorithm 4 with its residual in double-float (0, the default) or
    native float64 (1); other values are rejected."""
    from paper_2109_10687_gb300 import binding as B
    if residual_prec == 0:
        assert B.qcd_solve_params_default().residual_prec == 0
        for bad in (2, -1):
            _, rc, _ = c1.lat.solve(c1_ref[0], tol=1e-10, residual_prec=bad, raise_on_error=False)
            assert rc == B.QCD_ERR_ARG
    b, x_ref = c1_ref
    x, rc, info = c1.lat.solve(b, tol=1e-10, sap_prec="half", inner_tol=1e-5, residual_prec=residual_prec)
    x = to_np(x)
    assert rc == 0
    assert true_resid(c1.op, x, b) < 1e-10
    assert rel_l2(x, x_ref) < 1e-8


@pytest.mark.parametrize("kappa,seed", [(0.12, 1001), (0.125, 1002), (0.126, 1003)])
def test_double_float_residual_bound(kappa, seed):
    """Algorithm 4 with its residual r = b - D x in double-float (two float32,
    about 48 significant bits, unit u = 2^-48): the residual the solver
    reports, and stops on, differs from the float64 residual of the same x
    (recomputed by the oracle) by at most the rounding of D x and of b:
    |r_df - r_64| / |b| <= n_t u |D|_max |x| / |b| + u, with n_t = 100 terms
    per component of D x (8 hops of 3x3 links, the clover blocks) and
    |D|_max = 3 (1 + 8 kappa |U| (1 +- gamma) and 1 + C, 16 kappa < 2.1);
    that is 300 u |x| / |b|.  At the tolerance 1e-10 this is a few 1e-12
    relative error in the stopping test, the same order as the float64
    residual's own rounding times the lattice's condition."""
    p = Problem((8, 8, 8, 8), (4, 4, 4, 4), eps=0.3, kappa=kappa, csw=1.0, seed=seed)
    try:
        b = gaussian_spinor(p.dims, seed + 1000)
        x, rc, info = p.lat.solve(b, tol=1e-10, sap_prec="half", inner_tol=1e-5, residual_prec=0)
        x = to_np(x)
        assert rc == 0
        r64 = true_resid(p.op, x, b)
        assert r64 < 1e-10
        u = 2.0 ** -48
        bound = u + 300 * u * np.linalg.norm(x.ravel()) / np.linalg.norm(b.ravel())
        assert abs(info.true_resid - r64) <= bound, (info.true_resid, r64, bound)
        # the native float64 residual of the same solve agrees with the oracle to its own rounding
        x1, rc1, info1 = p.lat.solve(b, tol=1e-10, sap_prec="half", inner_tol=1e-5, residual_prec=1)
        assert rc1 == 0 and abs(info1.true_resid - true_resid(p.op, to_np(x1), b)) <= bound
    finally:
        p.close()


@pytest.mark.parametrize("factor", [1e-30, 1e25])
def test_double_float_residual_far_from_unit_sources(c1, c1_ref, factor):
    """The double-float residual (the default) keeps b, x and r scaled by a
    power of two that brings b's components to order one, so sources far
    outside float32's comfortable range solve as well: b times 1e-30 (whose
    residual at 1e-10 would be below float32's smallest normal number) and
    times 1e25.  x scales with b exactly; the oracle's residual of x is below
    1e-10 and agrees with the reported one."""
    b, x_ref = c1_ref
    bs = b * factor
    x, rc, info = c1.lat.solve(bs, tol=1e-10, sap_prec="half", inner_tol=1e-5)
    x = to_np(x)
    assert rc == 0
    r = true_resid(c1.op, x, bs)
    assert r < 1e-10 and abs(info.true_resid - r) <= 1e-12, (r, info.true_resid)
    assert rel_l2(x / factor, x_ref) < 1e-8


@pytest.mark.parametrize("use_graph", [0, 2])
@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, -1])
def test_solve_with_each_sap_kernel_shape(c1, c1_ref, shape, use_graph):
    """The solve with each shape of the SAP block kernel (one or two sites
    per thread, one CTA per right-hand side, M_SAP in one launch with or
    without staggered CTAs, or the autotuned one), with a host loop and with
    the device-side graph loop, reaches the float64 true residual 1e-10
    recomputed by the oracle."""
    from paper_2109_10687_gb300 import binding as B
    b, x_ref = c1_ref
    try:
        B.qcd_set_sap_shape(c1.lat.ctx, shape)
        x, rc, info = c1.lat.solve(b, tol=1e-10, sap_prec="half", inner_tol=1e-5, use_graph=use_graph)
    finally:
        B.qcd_set_sap_shape(c1.lat.ctx, -1)
    assert rc == 0
    assert true_resid(c1.op, to_np(x), b) < 1e-10
    assert rel_l2(to_np(x), x_ref) < 1e-8


def test_solve_host_buffers(c1, c1_ref):
    b, x_ref = c1_ref
    x, rc, info = c1.lat.solve(b, host=True, tol=1e-10)
    assert rc == 0 and isinstance(x, np.ndarray)
    assert true_resid(c1.op, x, b) < 1e-10


def test_algorithm5_iterates_match_oracle(c1):
    """Three iterations of Algorithm 5 inside one outer step, compared with the
    oracle's literal Algorithm 5 (x = M_SAP y) after three iterations."""
    b = gaussian_spinor(c1.dims, 2002)
    x, rc, info = c1.lat.solve(b, tol=1e-14, inner_tol=1e-30, max_outer=1, max_inner=3, n_sap=2, n_jac=3,
                               raise_on_error=False)
    assert info.inner_iters == 3 and info.outer_iters == 1
    bn = np.linalg.norm(b.ravel())
    bp = c1.op.apply_cinv(b / bn)
    x_or, _, it, status = solvers.bicgstab_precdd(c1.op, bp, 2, 3, 1e-30, 3)
    assert it == 3
    assert rel_l2(to_np(x), bn * x_or) < 2e-5


@pytest.mark.parametrize("use_graph", [0, 2])
def test_batched_point_sources(c1, use_graph):
    """Several spin-colour point sources in one batched solve (the device-side
    graph loop runs until the last right-hand side has converged)."""
    srcs = np.stack([point_source(c1.dims, c, s) for c, s in ((0, 0), (1, 2), (2, 3))])
    x, rc, info = c1.lat.solve(srcs, nrhs=3, tol=1e-10, use_graph=use_graph, sap_prec="half_gauge",
                               inner_tol=1e-5)
    x = to_np(x)
    assert rc == 0
    for r in range(3):
        assert true_resid(c1.op, x[r], srcs[r]) < 1e-10


def test_graph_loop_iteration_limit(c1):
    """The device-side loop stops at max_inner and reports it."""
    from paper_2109_10687_gb300 import binding as B
    b = gaussian_spinor(c1.dims, 2005)
    x, rc, info = c1.lat.solve(b, tol=1e-12, max_outer=1, max_inner=2, use_graph=2, raise_on_error=False)
    assert rc == B.QCD_ERR_NOT_CONVERGED
    assert info.inner_iters == 2


def test_zero_source(c1):
    z = np.zeros(c1.lat.site_shape + (3, 4), dtype=np.complex128)
    x, rc, info = c1.lat.solve(z, tol=1e-10)
    assert rc == 0 and np.abs(to_np(x)).max() == 0 and info.outer_iters == 0


def test_nonfinite_source_reports_status(c1):
    from paper_2109_10687_gb300 import binding as B
    b = gaussian_spinor(c1.dims, 2003)
    b[1, 2, 3, 4, 0, 0] = np.nan
    x, rc, info = c1.lat.solve(b, tol=1e-10, raise_on_error=False)
    assert rc == B.QCD_ERR_NONFINITE


def test_iteration_limit_reports_status(c1):
    from paper_2109_10687_gb300 import binding as B
    b = gaussian_spinor(c1.dims, 2004)
    x, rc, info = c1.lat.solve(b, tol=1e-12, max_outer=1, max_inner=1, raise_on_error=False)
    assert rc == B.QCD_ERR_NOT_CONVERGED
    assert info.outer_iters == 1


def test_resume_from_guess(c1, c1_ref):
    """A solve started from a previous iterate (x_is_guess) needs fewer steps."""
    b, x_ref = c1_ref
    x0, rc, _ = c1.lat.solve(b, tol=1e-6)
    from paper_2109_10687_gb300 import binding as B
    p = B.qcd_solve_params_default()
    p.x_is_guess = 1
    p.tol = 1e-10
    import torch
    src = torch.view_as_real(torch.from_numpy(b).cuda()).contiguous()
    out = torch.view_as_real(x0.contiguous()).contiguous().clone()
    rc, info = B.qcd_solve(c1.lat.ctx, out, src, 1, p)
    assert rc == 0
    assert true_resid(c1.op, to_np(torch.view_as_complex(out)), b) < 1e-10


def test_solve_full_size_sampled_32x4():
    """The 32^4 benchmark workload (same gauge recipe, seeds and parameters)
    solved in the launch configuration the benchmark times: float16-storage
    SAP, the inner loop as one graph with a conditional while node, float64
    defect correction.  The residual b - D x is recomputed on 64 sampled sites
    by the site-by-site float64 oracle, independently of the library's own D."""
    from oracle import pointwise
    dims = (32, 32, 32, 32)
    p = Problem(dims, (4, 4, 4, 4), eps=0.3, kappa=0.125, csw=1.0, seed=1001, oracle=False)
    try:
        b = gaussian_spinor(dims, 2001)
        x, rc, info = p.lat.solve(b, tol=1e-10, inner_tol=1e-5, n_sap=4, n_jac=4, sap_prec="half", use_graph=2)
        x = to_np(x)
        assert rc == 0 and info.true_resid < 1e-10
        rng = np.random.default_rng(7)
        num = den = 0.0
        for _ in range(64):
            c = tuple(int(rng.integers(0, dims[mu])) for mu in range(4))
            r = b[c[3], c[2], c[1], c[0]] - pointwise.D_at(p.u, x, c, 0.125, 1.0, p.gammas, -1)
            num += np.sum(np.abs(r) ** 2)
            den += np.sum(np.abs(b[c[3], c[2], c[1], c[0]]) ** 2)
        # a 64-site sample of a residual whose global relative norm is < 1e-10
        assert np.sqrt(num / den) < 1e-8
    finally:
        p.close()


@pytest.mark.parametrize("sap_prec", ["single", "half"])
def test_fgmres_outer_to_1e10(c1, c1_ref, sap_prec):
    """Flexible GMRES(4) as the outer iteration, the inner SAP-BiCGStab solve
    as its varying preconditioner: same true residual and solution bars as
    the defect correction of Algorithm 4."""
    b, x_ref = c1_ref
    x, rc, info = c1.lat.solve(b, tol=1e-10, inner_tol=1e-5, sap_prec=sap_prec, outer_restart=4, use_graph=2)
    x = to_np(x)
    assert rc == 0 and info.true_resid < 1e-10
    assert true_resid(c1.op, x, b) < 1e-10
    assert rel_l2(x, x_ref) < 1e-8


def test_fgmres_needs_no_more_outer_steps_than_defect_correction(c1, c1_ref):
    """With a loose inner tolerance the defect correction restarts from the
    bare residual every step, while flexible GMRES combines all earlier
    directions: it takes at most as many outer steps."""
    b, _ = c1_ref
    _, rc_d, info_d = c1.lat.solve(b, tol=1e-10, inner_tol=1e-2, sap_prec="single", max_outer=60)
    _, rc_f, info_f = c1.lat.solve(b, tol=1e-10, inner_tol=1e-2, sap_prec="single", max_outer=60, outer_restart=16)
    assert rc_d == 0 and rc_f == 0
    assert info_f.true_resid < 1e-10
    assert info_f.outer_iters <= info_d.outer_iters


def test_fgmres_rejects_multi_rhs(c1):
    from paper_2109_10687_gb300 import binding as B
    srcs = np.stack([point_source(c1.dims, 0, 0), point_source(c1.dims, 1, 1)])
    _, rc, _ = c1.lat.solve(srcs, nrhs=2, outer_restart=4, raise_on_error=False)
    assert rc == B.QCD_ERR_ARG


@pytest.fixture(scope="module")
def mixed_domains():
    """8x8x4x8 with 2x4x2x4 domains and periodic t: the generic (any domain
    shape) SAP kernel instead of the staged 4^4 one."""
    p = Problem((8, 8, 4, 8), (2, 4, 2, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1021, bc_t=1)
    yield p
    p.close()


@pytest.mark.parametrize("sap_prec", ["single", "half", "half_gauge"])
@pytest.mark.parametrize("use_graph", [0, 2])
def test_solve_generic_domains(mixed_domains, sap_prec, use_graph):
    b = gaussian_spinor(mixed_domains.dims, 2021)
    x, rc, info = mixed_domains.lat.solve(b, tol=1e-10, inner_tol=1e-5, sap_prec=sap_prec, use_graph=use_graph)
    x = to_np(x)
    assert rc == 0 and info.true_resid < 1e-10
    assert true_resid(mixed_domains.op, x, b) < 1e-10


@pytest.mark.parametrize("sap_prec", ["single", "half_gauge"])
def test_solve_on_paper_sap_domains(sap_prec):
    """The solve with the paper's algorithm parameters (n_sap 4, n_jac 2) on
    its 16x6x4x3 SAP domains (Sec. 4.3), fields stored in 4x2x2x1 blocks:
    float64 true residual below 1e-10, recomputed by the oracle."""
    from paper_2109_10687_gb300 import binding as B
    p = Problem((32, 12, 8, 6), (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1131)
    try:
        B.qcd_set_sap_domain(p.lat.ctx, (16, 6, 4, 3))
        b = gaussian_spinor(p.dims, 2131)
        for use_graph in (0, 2):
            x, rc, info = p.lat.solve(b, tol=1e-10, inner_tol=1e-6 if sap_prec == "single" else 1e-5, n_sap=4,
                                      n_jac=2, sap_prec=sap_prec, use_graph=use_graph)
            assert rc == 0 and true_resid(p.op, to_np(x), b) < 1e-10
        # half (float16 vectors) is not offered on general domains
        _, rc, _ = p.lat.solve(b, tol=1e-10, sap_prec="half", raise_on_error=False)
        assert rc == B.QCD_ERR_ARG
    finally:
        p.close()

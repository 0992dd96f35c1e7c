"""Ragged batches: several lattices of different sizes, gauge fields and
kappa in one operator launch and one batched solve, against the oracle."""

import numpy as np
import pytest
import torch

from gpu_util import Problem, rel_l2, to_np
from lattice_inputs import gaussian_spinor

pytestmark = pytest.mark.gpu

LATTICES = [((8, 8, 8, 8), 0.120, 5000), ((16, 8, 8, 8), 0.118, 5001), ((8, 16, 8, 16), 0.122, 5002),
            ((8, 8, 16, 8), 0.115, 5003)]


@pytest.fixture(scope="module")
def batch():
    from paper_2109_10687_gb300 import binding as B
    probs = [Problem(d, (4, 4, 4, 4), eps=0.3, kappa=k, csw=1.0, seed=s) for d, k, s in LATTICES]
    bt = B.qcd_batch_create([p.lat.ctx for p in probs])
    yield probs, bt
    B.qcd_batch_destroy(bt)
    for p in probs:
        p.close()


def test_batch_apply_D_one_launch(batch):
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    xs = [gaussian_spinor(p.dims, 6000 + i) for i, p in enumerate(probs)]
    ins = [p.lat.to_internal(x, "single") for p, x in zip(probs, xs)]
    outs = [p.lat.field("single") for p in probs]
    n0 = B.qcd_launch_count(probs[0].lat.ctx)
    for dagger in (0, 1):
        B.qcd_batch_apply_D(bt, outs, ins, dagger)
        for p, x, o in zip(probs, xs, outs):
            got = to_np(p.lat.to_canonical(o, "single"))
            ref = p.op.Ddag(x) if dagger else p.op.D(x)
            assert rel_l2(got, ref) <= 1e-6
    # one kernel per batched application, counted on the first context
    assert B.qcd_launch_count(probs[0].lat.ctx) - n0 == 2 + 2  # 2 applies + 2 exports on ctx 0


def test_batch_solve(batch):
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    bs = [torch.view_as_real(torch.from_numpy(gaussian_spinor(p.dims, 6100 + i))).cuda().contiguous()
          for i, p in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    params = B.qcd_solve_params_default()
    params.sap_prec = B.PREC_HALF
    params.inner_tol = 1e-5
    rc, infos = B.qcd_batch_solve(bt, xs, bs, params)
    assert rc == 0
    for p, x, b, info in zip(probs, xs, bs, infos):
        xn = to_np(torch.view_as_complex(x))
        bn = to_np(torch.view_as_complex(b))
        r = np.linalg.norm((bn - p.op.D(xn)).ravel()) / np.linalg.norm(bn.ravel())
        assert r < 1e-10 and info.true_resid < 1e-10


def _solve_batch(bt, probs, seed, shared=True, **kw):
    from paper_2109_10687_gb300 import binding as B
    bs = [torch.view_as_real(torch.from_numpy(gaussian_spinor(p.dims, seed + i))).cuda().contiguous()
          for i, p in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    params = B.qcd_solve_params_default()
    params.inner_tol = 1e-5
    for k, v in kw.items():
        setattr(params, k, v)
    B.qcd_batch_set_shared(bt, shared)
    try:
        rc, infos = B.qcd_batch_solve(bt, xs, bs, params, raise_on_error=False)
    finally:
        B.qcd_batch_set_shared(bt, True)
    return rc, infos, xs, bs


def _oracle_resid(p, x, b):
    xn = to_np(torch.view_as_complex(x))
    bn = to_np(torch.view_as_complex(b))
    return np.linalg.norm((bn - p.op.D(xn)).ravel()) / np.linalg.norm(bn.ravel())


@pytest.mark.parametrize("sap_prec,use_graph", [("half", 2), ("single", 2), ("half_gauge", 0)])
def test_batch_solve_shared_launches(batch, sap_prec, use_graph):
    """The shared-launch ragged solve: every lattice's SAP half-sweeps, A and
    D applications and BLAS-1 steps in launches over all four lattices.
    Each lattice's float64 true residual, recomputed by the oracle, is below
    1e-10; the library's per-lattice report agrees with it; each lattice's
    iteration count is its own (close to its solve alone)."""
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    prec = {"half": B.PREC_HALF, "single": B.PREC_SINGLE, "half_gauge": B.PREC_HALF_GAUGE}[sap_prec]
    n0 = B.qcd_launch_count(probs[0].lat.ctx)
    rc, infos, xs, bs = _solve_batch(bt, probs, 6200, sap_prec=prec, use_graph=use_graph)
    launches = B.qcd_launch_count(probs[0].lat.ctx) - n0
    assert rc == 0, B.lib().qcd_batch_last_error(bt)
    u = 2.0 ** -48
    for i, (p, x, b, info) in enumerate(zip(probs, xs, bs, infos)):
        r = _oracle_resid(p, x, b)
        assert r < 1e-10 and info.true_resid < 1e-10, (i, r, info.true_resid)
        # the default residual's D is double-float: within its bound of the float64 residual
        xb = float(torch.linalg.vector_norm(x) / torch.linalg.vector_norm(b))
        assert abs(r - info.true_resid) <= u + 300 * u * xb, (i, r, info.true_resid)
        assert info.status == 0 and info.outer_iters >= 1 and info.inner_iters >= 1
        # the same lattice solved alone takes about as many iterations
        _, _, alone = p.lat.solve(to_np(torch.view_as_complex(b)), tol=1e-10, inner_tol=1e-5, sap_prec=prec,
                                  use_graph=use_graph)
        assert abs(alone.inner_iters - info.inner_iters) <= 2 + info.inner_iters // 5, (i, alone.inner_iters,
                                                                                      info.inner_iters)
    # every launch serves the four lattices: an iteration is about 28 launches
    # (2 x (10 SAP half-sweeps + A) + 6 others) for all of them together,
    # about half of what one lattice's iterations alone would launch over the
    # four solves
    assert launches < 14 * sum(i.inner_iters for i in infos) + 60, launches


@pytest.mark.parametrize("residual_prec", [0, 1])
def test_batch_solve_residual_precisions(batch, residual_prec):
    """The shared-launch solve with the residual's D in double-float (0, the
    default: each lattice's x copied with the power of two of its |b|^2,
    one launch over all lattices, the result rounded to float64) and in
    float64 (1): every lattice's oracle residual below 1e-10; the reported
    residual equals the oracle's to float64 rounding (1) or within the
    double-float bound (0)."""
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    rc, infos, xs, bs = _solve_batch(bt, probs, 6250, sap_prec=B.PREC_HALF, residual_prec=residual_prec)
    assert rc == 0
    u = 2.0 ** -48
    for p, x, b, info in zip(probs, xs, bs, infos):
        r = _oracle_resid(p, x, b)
        assert r < 1e-10
        xb = float(torch.linalg.vector_norm(x) / torch.linalg.vector_norm(b))
        tol = 1e-12 if residual_prec == 1 else u + 300 * u * xb
        assert abs(r - info.true_resid) <= tol, (residual_prec, r, info.true_resid)


def test_batch_solve_lattices_stop_separately(batch):
    """Each lattice stops on its own: a zero source needs no outer step and
    returns x = 0 (whatever x held) while the others iterate; a source 1e-30
    times the others' size (whose residual at 1e-10 lies below float32's
    range, so the double-float D must work on its scaled copy) still
    reaches the relative tolerance 1e-10."""
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    bs = [torch.view_as_real(torch.from_numpy(gaussian_spinor(p.dims, 6300 + i))).cuda().contiguous()
          for i, p in enumerate(probs)]
    bs[1] = bs[1] * 1e-30
    bs[2] = torch.zeros_like(bs[2])
    xs = [torch.full_like(b, 7.0) for b in bs]
    params = B.qcd_solve_params_default()
    params.inner_tol = 1e-5
    params.sap_prec = B.PREC_HALF
    rc, infos = B.qcd_batch_solve(bt, xs, bs, params)
    assert rc == 0
    assert infos[2].outer_iters == 0 and infos[2].inner_iters == 0 and float(xs[2].abs().max()) == 0.0
    for i in (0, 1, 3):
        assert _oracle_resid(probs[i], xs[i], bs[i]) < 1e-10


def test_batch_solve_resume_from_guess(batch):
    """x_is_guess: a second shared-launch solve started from the first one's
    solution needs no outer step."""
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    rc, infos, xs, bs = _solve_batch(bt, probs, 6400, sap_prec=B.PREC_HALF)
    assert rc == 0
    params = B.qcd_solve_params_default()
    params.x_is_guess = 1
    rc2, infos2 = B.qcd_batch_solve(bt, xs, bs, params)
    assert rc2 == 0 and all(i.outer_iters == 0 for i in infos2)
    for p, x, b in zip(probs, xs, bs):
        assert _oracle_resid(p, x, b) < 1e-10


def test_batch_solve_concurrent_form_agrees(batch):
    """The concurrent per-lattice form (qcd_batch_set_shared(batch, 0)) meets
    the same bar on the same sources."""
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    rc, infos, xs, bs = _solve_batch(bt, probs, 6500, shared=False, sap_prec=B.PREC_HALF)
    assert rc == 0
    for p, x, b in zip(probs, xs, bs):
        assert _oracle_resid(p, x, b) < 1e-10


def test_batch_solve_iteration_limit_reports_status(batch):
    from paper_2109_10687_gb300 import binding as B
    probs, bt = batch
    rc, infos, xs, bs = _solve_batch(bt, probs, 6600, sap_prec=B.PREC_HALF, max_outer=1, max_inner=2)
    assert rc == B.QCD_ERR_NOT_CONVERGED
    assert all(i.status == B.QCD_ERR_NOT_CONVERGED and i.outer_iters == 1 for i in infos)


def test_batch_solve_follows_a_new_kappa(batch):
    """After a lattice's kappa changes (qcd_set_params + qcd_build_clover), the
    next shared-launch solve uses the new operator: the oracle residual with
    the new kappa is below 1e-10 for every lattice."""
    from paper_2109_10687_gb300 import binding as B
    from oracle.dirac import CloverWilson
    probs, bt = batch
    p0 = probs[0]
    old_kappa = p0.kappa
    new_kappa = 0.110
    try:
        B.qcd_set_params(p0.lat.ctx, new_kappa, p0.csw)
        B.qcd_build_clover(p0.lat.ctx)
        rc, infos, xs, bs = _solve_batch(bt, probs, 6700, sap_prec=B.PREC_HALF)
        assert rc == 0
        op_new = CloverWilson(p0.u, new_kappa, p0.csw, p0.gammas, bc_t=-1)
        xn = to_np(torch.view_as_complex(xs[0]))
        bn = to_np(torch.view_as_complex(bs[0]))
        assert np.linalg.norm((bn - op_new.D(xn)).ravel()) / np.linalg.norm(bn.ravel()) < 1e-10
        for p, x, b in zip(probs[1:], xs[1:], bs[1:]):
            assert _oracle_resid(p, x, b) < 1e-10
    finally:
        B.qcd_set_params(p0.lat.ctx, old_kappa, p0.csw)
        B.qcd_build_clover(p0.lat.ctx)


def test_batch_solve_periodic_time_and_paper_basis():
    """The shared-launch solve with periodic time (bc_t = +1) and with fields in
    the paper's gamma basis (rotated on import and export per lattice): every
    lattice's oracle residual below 1e-10."""
    from paper_2109_10687_gb300 import binding as B
    for bc_t, basis in ((+1, "chiral"), (-1, "paper")):
        probs = [Problem(d, (4, 4, 4, 4), eps=0.3, kappa=k, csw=1.0, seed=s + 50, bc_t=bc_t, basis=basis)
                 for d, k, s in LATTICES[:3]]
        bt = B.qcd_batch_create([p.lat.ctx for p in probs])
        try:
            rc, infos, xs, bs = _solve_batch(bt, probs, 6800, sap_prec=B.PREC_HALF)
            assert rc == 0
            for p, x, b in zip(probs, xs, bs):
                assert _oracle_resid(p, x, b) < 1e-10, (bc_t, basis)
        finally:
            B.qcd_batch_destroy(bt)
            for p in probs:
                p.close()

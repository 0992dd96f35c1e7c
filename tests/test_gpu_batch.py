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

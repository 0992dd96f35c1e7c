"""GPU parity of the SAP preconditioner (Algorithms 1-3) against the oracle's
literal Algorithms, float32 and float16 storage."""

import numpy as np
import pytest

from gpu_util import Problem, rel_l2, to_np
from oracle import sap

pytestmark = pytest.mark.gpu

CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4)),
    ((4, 4, 4, 8), (2, 2, 2, 2)),
    ((8, 8, 4, 8), (2, 4, 2, 4)),
    ((2, 2, 2, 2), (1, 1, 1, 1)),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])) + "_d" + "".join(map(str, c[1])))
def prob(request):
    dims, domain = request.param
    p = Problem(dims, domain, eps=0.3, kappa=0.12, csw=1.0, seed=1101)
    yield p
    p.close()


@pytest.mark.parametrize("n_sap,n_jac", [(0, 1), (1, 2), (4, 4)])
def test_msap_float32(prob, n_sap, n_jac):
    b = prob.source(2101)
    got = to_np(prob.lat.sap(b, n_sap, n_jac, "single"))
    ref = sap.msap(prob.op, b, n_sap, n_jac)
    assert rel_l2(got, ref) <= 1e-5


def test_am_sap_float32(prob):
    b = prob.source(2102)
    got = to_np(prob.lat.sap(b, 4, 4, "single", with_A=True))
    ref = sap.am_sap(prob.op, b, 4, 4)
    assert rel_l2(got, ref) <= 1e-5


def test_msap_float16_storage(prob):
    """float16 storage with per-site norms: an approximation of M_SAP at the
    level of half-precision rounding (2^-11 per stored value)."""
    b = prob.source(2103)
    got = to_np(prob.lat.sap(b, 4, 4, "half"))
    ref = sap.msap(prob.op, b, 4, 4)
    assert rel_l2(got, ref) <= 5e-3


def test_msap_float16_gauge_storage(prob):
    """float16 links and C_inv with float32 vectors: an approximation of M_SAP
    at the level of half-precision rounding of the operator."""
    b = prob.source(2105)
    got = to_np(prob.lat.sap(b, 4, 4, "half_gauge"))
    ref = sap.msap(prob.op, b, 4, 4)
    assert rel_l2(got, ref) <= 5e-3


def test_sap_reduces_residual(prob):
    """A M_SAP is close to the identity: |b - A M b| / |b| well below 1."""
    b = prob.source(2104)
    amb = to_np(prob.lat.sap(b, 4, 4, "single", with_A=True))
    assert rel_l2(amb, b) < 0.5


@pytest.fixture(scope="module")
def wide():
    """16x8x8x8 with 4^4 domains: four domains along x, so a domain's forward
    and backward neighbours differ (with two per direction they coincide)."""
    p = Problem((16, 8, 8, 8), (4, 4, 4, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1111)
    yield p
    p.close()


@pytest.mark.parametrize("sap_prec,tol", [("single", 1e-5), ("half_gauge", 5e-3), ("half", 5e-3)])
def test_msap_four_domains_per_direction(wide, sap_prec, tol):
    b = wide.source(2106)
    got = to_np(wide.lat.sap(b, 4, 4, sap_prec))
    ref = sap.msap(wide.op, b, 4, 4)
    assert rel_l2(got, ref) <= tol


@pytest.mark.parametrize("sap_prec", ["single", "half_gauge", "half"])
@pytest.mark.parametrize("with_A", [False, True])
def test_msap_multi_rhs_matches_single_rhs(wide, sap_prec, with_A):
    """Three right-hand sides through each launch (shared staging, one halo
    block per right-hand side): each result equals the single-rhs result bit
    for bit, and the oracle's within the storage's tolerance."""
    srcs = np.stack([wide.source(2110 + r) for r in range(3)])
    got = to_np(wide.lat.sap(srcs, 4, 4, sap_prec, with_A=with_A, nrhs=3))
    tol = 1e-5 if sap_prec == "single" else 5e-3
    for r in range(3):
        one = to_np(wide.lat.sap(srcs[r], 4, 4, sap_prec, with_A=with_A))
        assert np.array_equal(got[r], one), r
        ref = (sap.am_sap if with_A else sap.msap)(wide.op, srcs[r], 4, 4)
        assert rel_l2(got[r], ref) <= tol


@pytest.mark.parametrize("sap_prec", ["single", "half_gauge", "half"])
def test_sap_kernel_shapes_agree_bit_for_bit(wide, sap_prec):
    """The shapes of the SAP block kernel for 4^4 domains (one site per
    thread, two sites per thread, one CTA per domain and right-hand side) do
    the same arithmetic per site, so their M_SAP agree bit for bit, single and
    batched; all match the oracle's literal Algorithm 1 within the storage's
    tolerance.  With the shape left to the autotuner, the tuning report lists
    the SAP key and the shapes."""
    from paper_2109_10687_gb300 import binding as B
    ctx = wide.lat.ctx
    b = wide.source(2120)
    srcs = np.stack([wide.source(2121 + r) for r in range(2)])
    out = {}
    try:
        for shape in (0, 1, 2, 3, 4):
            B.qcd_set_sap_shape(ctx, shape)
            out[shape] = (to_np(wide.lat.sap(b, 4, 4, sap_prec)), to_np(wide.lat.sap(srcs, 4, 4, sap_prec, nrhs=2)))
        B.qcd_set_sap_shape(ctx, -1)
        tuned = to_np(wide.lat.sap(b, 4, 4, sap_prec))
        tuned2 = to_np(wide.lat.sap(srcs, 4, 4, sap_prec, nrhs=2))
    finally:
        B.qcd_set_sap_shape(ctx, -1)
    for shape in (1, 2, 3, 4):
        assert np.array_equal(out[0][0], out[shape][0])
        assert np.array_equal(out[0][1], out[shape][1])
    assert np.array_equal(tuned2, out[0][1])
    assert np.array_equal(tuned, out[0][0])
    tol = 1e-5 if sap_prec == "single" else 5e-3
    assert rel_l2(out[1][0], sap.msap(wide.op, b, 4, 4)) <= tol
    rep = B.qcd_tuning_report(ctx)
    line = [ln for ln in rep.splitlines() if ln.startswith("sap_staged_")]
    assert line and "256x1site" in line[0] and "128x2sites" in line[0] and "one_launch" in line[0]
    assert any("nrhs2" in ln and "256x1site_rhs_grid" in ln and "one_launch_staggered" in ln for ln in line)


@pytest.fixture(scope="module")
def cube8():
    """8^4 with 4^4 domains: eight domains per colour, so a one-launch M_SAP
    runs many more CTAs than a half-sweep has domains, and most items wait
    on their neighbours' flags."""
    p = Problem((8, 8, 8, 8), (4, 4, 4, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1131)
    yield p
    p.close()


@pytest.mark.parametrize("lattice", ["wide", "cube8"])
@pytest.mark.parametrize("sap_prec", ["single", "half_gauge", "half"])
@pytest.mark.parametrize("n_sap,n_jac", [(1, 1), (2, 4), (4, 4)])
def test_sap_one_launch_matches_per_launch(request, lattice, sap_prec, n_sap, n_jac):
    """M_SAP in one launch (shapes 3 and 4: resident CTAs taking (half-sweep,
    domain) items in order, each waiting for its eight neighbours' flags)
    does every domain's half-sweeps with the per-launch kernel's arithmetic
    in the same order of dependencies, so M_SAP and A M_SAP agree bit for bit
    with shape 0, for one and for three right-hand sides, and stay so on a
    second call (the counters and flags are cleared by the last CTA)."""
    from paper_2109_10687_gb300 import binding as B
    p = request.getfixturevalue(lattice)
    ctx = p.lat.ctx
    b = p.source(2140)
    srcs = np.stack([p.source(2141 + r) for r in range(3)])
    out = {}
    try:
        for shape in (0, 3, 4, 3):
            B.qcd_set_sap_shape(ctx, shape)
            out.setdefault(shape, []).append((to_np(p.lat.sap(b, n_sap, n_jac, sap_prec)),
                                              to_np(p.lat.sap(b, n_sap, n_jac, sap_prec, with_A=True)),
                                              to_np(p.lat.sap(srcs, n_sap, n_jac, sap_prec, nrhs=3))))
            assert B.qcd_device_status(ctx) == B.QCD_OK
    finally:
        B.qcd_set_sap_shape(ctx, -1)
    ref = out[0][0]
    for shape in (3, 4):
        for got in out[shape]:
            for g_, r_ in zip(got, ref):
                assert np.array_equal(g_, r_), (shape, lattice)
    tol = 1e-5 if sap_prec == "single" else 5e-3
    assert rel_l2(out[3][0][0], sap.msap(p.op, b, n_sap, n_jac)) <= tol


@pytest.mark.parametrize("hook,prec", [("staging", "half"), ("halo", "half_gauge")])
def test_one_launch_wait_timeout_is_reported_and_context_survives(cube8, hook, prec):
    """The one-launch M_SAP's failure path, without a GPU fault: a test hook
    makes the staging (or halo) wait expect 16 bytes that no copy brings.
    Every item that meets it gives up after half a second and records
    QCD_ERR_TIMEOUT; the other CTAs see the status, stop waiting for flags
    and leave; the last one clears the counters and flags.  With the hook
    cleared, the same context's next one-launch M_SAP is correct."""
    from paper_2109_10687_gb300 import binding as B
    ctx = cube8.lat.ctx
    b = cube8.source(2150)
    inj = B.INJECT_STAGING_WAIT if hook == "staging" else B.INJECT_HALO_WAIT
    try:
        B.qcd_set_sap_shape(ctx, 3)
        B.qcd_test_inject(ctx, inj)
        cube8.lat.sap(b, 1, 1, prec)
        assert B.qcd_device_status(ctx, reset=True) == B.QCD_ERR_TIMEOUT
        B.qcd_test_inject(ctx, B.INJECT_NONE)
        got = to_np(cube8.lat.sap(b, 4, 4, prec))
        assert B.qcd_device_status(ctx) == B.QCD_OK
        B.qcd_set_sap_shape(ctx, 0)
        ref = to_np(cube8.lat.sap(b, 4, 4, prec))
        assert np.array_equal(got, ref)
    finally:
        B.qcd_test_inject(ctx, B.INJECT_NONE)
        B.qcd_device_status(ctx, reset=True)
        B.qcd_set_sap_shape(ctx, -1)


def test_sap_shape_rejects_unknown_value(wide):
    from paper_2109_10687_gb300 import binding as B
    assert B.lib().qcd_set_sap_shape(wide.lat.ctx, 5) == B.QCD_ERR_ARG
    assert B.lib().qcd_set_sap_shape(wide.lat.ctx, -2) == B.QCD_ERR_ARG


def test_sap_apply_nrhs_rejects_bad_count(wide):
    from paper_2109_10687_gb300 import binding as B
    a = wide.lat.field("single", 1)
    o = wide.lat.field("single", 1)
    rc = B.lib().qcd_sap_apply_nrhs(wide.lat.ctx, B._ptr(o), B._ptr(a), 0, 4, 4, B.PREC_SINGLE, 0, None)
    assert rc == B.QCD_ERR_ARG


def test_staging_wait_timeout_is_reported_and_context_survives():
    """Failure path of the SAP block kernel's bounded wait, without a GPU fault:
    the test hook makes the wait expect 16 bytes that no copy brings, so it
    runs out (half a second), the kernel records QCD_ERR_TIMEOUT, waits once
    more (bounded) and returns.  The status reaches the host, a solve reports
    it, and with the hook cleared the same context computes M_SAP correctly."""
    from paper_2109_10687_gb300 import binding as B
    p = Problem((8, 8, 8, 8), (4, 4, 4, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1101)
    try:
        b = p.source(2106)
        B.qcd_test_inject(p.lat.ctx, B.INJECT_STAGING_WAIT)
        p.lat.sap(b, 0, 1, "half")
        assert B.qcd_device_status(p.lat.ctx, reset=True) == B.QCD_ERR_TIMEOUT
        _, rc, _ = p.lat.solve(b, tol=1e-10, n_sap=0, n_jac=1, max_inner=1, max_outer=1, sap_prec="half",
                               raise_on_error=False)
        assert rc == B.QCD_ERR_TIMEOUT
        B.qcd_test_inject(p.lat.ctx, B.INJECT_NONE)
        B.qcd_device_status(p.lat.ctx, reset=True)
        got = to_np(p.lat.sap(b, 4, 4, "half"))
        assert B.qcd_device_status(p.lat.ctx) == B.QCD_OK
        assert rel_l2(got, sap.msap(p.op, b, 4, 4)) <= 5e-3
    finally:
        p.close()


def test_halo_wait_timeout_is_reported_and_context_survives():
    """The same failure path for the wait on the face-halo copy, which only
    launches with a surface term make (here the O half-sweep)."""
    from paper_2109_10687_gb300 import binding as B
    p = Problem((8, 8, 8, 8), (4, 4, 4, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1101)
    try:
        b = p.source(2107)
        B.qcd_test_inject(p.lat.ctx, B.INJECT_HALO_WAIT)
        p.lat.sap(b, 0, 1, "half_gauge")
        assert B.qcd_device_status(p.lat.ctx, reset=True) == B.QCD_ERR_TIMEOUT
        B.qcd_test_inject(p.lat.ctx, B.INJECT_NONE)
        got = to_np(p.lat.sap(b, 4, 4, "half_gauge"))
        assert B.qcd_device_status(p.lat.ctx) == B.QCD_OK
        assert rel_l2(got, sap.msap(p.op, b, 4, 4)) <= 5e-3
    finally:
        p.close()


@pytest.fixture(scope="module")
def paper_domains():
    """32x12x8x6 stored in 4x2x2x1 blocks, with the SAP on the paper's
    16x6x4x3 domains (Sec. 4.3, Tables 2-3): two domains per direction."""
    from paper_2109_10687_gb300 import binding as B
    p = Problem((32, 12, 8, 6), (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1121, oracle=False)
    B.qcd_set_sap_domain(p.lat.ctx, (16, 6, 4, 3))
    from oracle.dirac import CloverWilson
    p.op = CloverWilson(p.u, 0.12, 1.0, p.gammas, bc_t=-1, domain=(16, 6, 4, 3))
    yield p
    p.close()


@pytest.mark.parametrize("n_sap,n_jac", [(0, 1), (4, 2)])
def test_msap_paper_domains_float32(paper_domains, n_sap, n_jac):
    """M_SAP on non-power-of-two domains against the oracle's literal
    Algorithm 1 on the same domains, at the paper's n_sap 4, n_jac 2."""
    b = paper_domains.source(2130)
    got = to_np(paper_domains.lat.sap(b, n_sap, n_jac, "single"))
    ref = sap.msap(paper_domains.op, b, n_sap, n_jac)
    assert rel_l2(got, ref) <= 1e-5


def test_msap_paper_domains_float16_gauge(paper_domains):
    b = paper_domains.source(2131)
    got = to_np(paper_domains.lat.sap(b, 4, 2, "half_gauge"))
    assert rel_l2(got, sap.msap(paper_domains.op, b, 4, 2)) <= 5e-3


def test_am_sap_and_nrhs_paper_domains(paper_domains):
    srcs = np.stack([paper_domains.source(2132 + r) for r in range(2)])
    got = to_np(paper_domains.lat.sap(srcs, 1, 2, "single", with_A=True, nrhs=2))
    for r in range(2):
        assert rel_l2(got[r], sap.am_sap(paper_domains.op, srcs[r], 1, 2)) <= 1e-5


def test_msap_general_domains_four_per_direction():
    """8x6x4x3 domains on 32x12x8x6: four domains along x, so a domain's
    forward and backward neighbours differ."""
    from paper_2109_10687_gb300 import binding as B
    from oracle.dirac import CloverWilson
    p = Problem((32, 12, 8, 6), (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1122, oracle=False)
    try:
        B.qcd_set_sap_domain(p.lat.ctx, (8, 6, 4, 3))
        op = CloverWilson(p.u, 0.12, 1.0, p.gammas, bc_t=-1, domain=(8, 6, 4, 3))
        b = p.source(2133)
        assert rel_l2(to_np(p.lat.sap(b, 2, 2, "single")), sap.msap(op, b, 2, 2)) <= 1e-5
        # back to the storage domains: the shared-nothing generic kernel on 4x2x2x1
        B.qcd_set_sap_domain(p.lat.ctx, None)
        op.set_domain((4, 2, 2, 1))
        assert rel_l2(to_np(p.lat.sap(b, 1, 2, "single")), sap.msap(op, b, 1, 2)) <= 1e-5
    finally:
        p.close()


def test_large_domains_need_the_cluster_kernel():
    """A 16x6x4x6 domain (2304 sites, above the one-CTA kernel's 1152) is
    accepted, since its six time slices of 384 sites fit the cluster
    kernel; the SAP then runs only with float16 links and C_inv on the
    cluster shape: float32, and the one-CTA shape, are QCD_ERR_ARG; a
    domain that fits neither kernel (16x6x4x12: 12 slices) is rejected."""
    from paper_2109_10687_gb300 import binding as B
    p = Problem((32, 12, 8, 12), (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1153, oracle=False)
    try:
        ctx = p.lat.ctx
        assert B.lib().qcd_set_sap_domain(ctx, (B.ctypes.c_int * 4)(16, 6, 4, 12)) == B.QCD_ERR_ARG
        B.qcd_set_sap_domain(ctx, (16, 6, 4, 6))
        a = p.lat.to_internal(p.source(2170), "single")
        o = p.lat.field("single")
        assert B.lib().qcd_sap_apply(ctx, B._ptr(o), B._ptr(a), 1, 1, B.PREC_SINGLE, 0, None) == B.QCD_ERR_ARG
        B.qcd_set_sap_shape(ctx, 1)
        assert B.lib().qcd_sap_apply(ctx, B._ptr(o), B._ptr(a), 1, 1, B.PREC_HALF_GAUGE, 0, None) == B.QCD_ERR_ARG
        B.qcd_set_sap_shape(ctx, -1)
        assert B.lib().qcd_sap_apply(ctx, B._ptr(o), B._ptr(a), 1, 1, B.PREC_HALF_GAUGE, 0, None) == B.QCD_OK
    finally:
        p.close()


def test_sap_domain_rejections(paper_domains):
    from paper_2109_10687_gb300 import binding as B
    ctx = paper_domains.lat.ctx
    assert B.lib().qcd_set_sap_domain(ctx, (B.ctypes.c_int * 4)(16, 6, 4, 5)) == B.QCD_ERR_ARG
    assert B.lib().qcd_set_sap_domain(ctx, (B.ctypes.c_int * 4)(32, 12, 8, 3)) == B.QCD_ERR_ARG  # 2 d must divide L
    a = paper_domains.lat.field("single")
    o = paper_domains.lat.field("single")
    rc = B.lib().qcd_sap_apply(ctx, B._ptr(o), B._ptr(a), 1, 1, B.PREC_HALF, 0, None)
    assert rc == B.QCD_ERR_ARG


def _half_round(a):
    return a.real.astype(np.float16).astype(np.float64) + 1j * a.imag.astype(np.float16).astype(np.float64)


@pytest.mark.parametrize("dims,sdom", [((32, 12, 8, 6), (16, 6, 4, 3)), ((32, 12, 8, 6), (8, 6, 4, 3)),
                                       ((32, 12, 8, 12), (8, 6, 4, 6)), ((32, 12, 8, 12), (16, 6, 4, 6))])
def test_cluster_sap_kernel_on_general_domains(dims, sdom):
    """The thread-block-cluster SAP kernel (one CTA per time slice of a
    domain, the t hops between slices through distributed shared memory,
    float16 links and C_inv staged in shared memory) gives M_SAP bit for bit
    equal to the one-CTA-per-domain kernel (same float16 operator, same
    arithmetic order), and matches the oracle's literal Algorithm 1 on the
    same float16-rounded links and C_inv to 1e-5, with 3 and 6 slices per
    domain.  The paper's 16x6x4x6 domain (2304 sites) fits only the cluster
    kernel: there the autotuned run is the cluster kernel's."""
    import copy
    from paper_2109_10687_gb300 import binding as B
    from oracle.dirac import CloverWilson
    p = Problem(dims, (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1151, oracle=False)
    try:
        B.qcd_set_sap_domain(p.lat.ctx, sdom)
        op = CloverWilson(p.u, 0.12, 1.0, p.gammas, bc_t=-1, domain=sdom)
        op16 = copy.copy(op)
        op16.u = _half_round(op.u)
        op16.cinv = _half_round(op.cinv)
        b = p.source(2160)
        one_cta = int(np.prod(sdom)) <= 1152
        out = {}
        for shape in ((0, 1) if one_cta else (0,)):
            B.qcd_set_sap_shape(p.lat.ctx, shape)
            out[shape] = to_np(p.lat.sap(b, 2, 2, "half_gauge"))
        B.qcd_set_sap_shape(p.lat.ctx, -1)
        if one_cta:
            assert np.array_equal(out[0], out[1])
        assert rel_l2(out[0], sap.msap(op16, b, 2, 2)) <= 1e-5
        rep = B.qcd_tuning_report(p.lat.ctx)
        tuned = to_np(p.lat.sap(b, 2, 2, "half_gauge"))
        assert np.array_equal(tuned, out[0])
        if one_cta:
            assert "cluster_per_domain" in B.qcd_tuning_report(p.lat.ctx) or "cluster_per_domain" in rep
    finally:
        p.close()


def test_cluster_sap_wait_timeout_is_reported_and_context_survives():
    """The failure path of the cluster kernel's bounded staging wait, without a
    GPU fault: the test hook makes every CTA's wait expect 16 bytes that no
    copy brings; the CTAs of a cluster agree through distributed shared memory
    that a wait gave up, record QCD_ERR_TIMEOUT and leave together; the status
    reaches the host and the same context then computes M_SAP correctly."""
    from paper_2109_10687_gb300 import binding as B
    p = Problem((32, 12, 8, 6), (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1152)
    try:
        B.qcd_set_sap_domain(p.lat.ctx, (16, 6, 4, 3))
        B.qcd_set_sap_shape(p.lat.ctx, 0)
        b = p.source(2161)
        B.qcd_test_inject(p.lat.ctx, B.INJECT_STAGING_WAIT)
        p.lat.sap(b, 0, 1, "half_gauge")
        assert B.qcd_device_status(p.lat.ctx, reset=True) == B.QCD_ERR_TIMEOUT
        B.qcd_test_inject(p.lat.ctx, B.INJECT_NONE)
        got = to_np(p.lat.sap(b, 1, 2, "half_gauge"))
        assert B.qcd_device_status(p.lat.ctx) == B.QCD_OK
        from oracle.dirac import CloverWilson
        op = CloverWilson(p.u, 0.12, 1.0, p.gammas, bc_t=-1, domain=(16, 6, 4, 3))
        assert rel_l2(got, sap.msap(op, b, 1, 2)) <= 5e-3
    finally:
        p.close()


def test_cluster_sap_kernel_periodic_time():
    """The cluster kernel with periodic time (bc_t = +1; the boundary sign
    sits on the surface hops across t = Lt - 1 <-> 0): bit for bit equal to the
    one-CTA kernel and within 1e-5 of the oracle on the rounded operator."""
    import copy
    from paper_2109_10687_gb300 import binding as B
    from oracle.dirac import CloverWilson
    p = Problem((32, 12, 8, 6), (4, 2, 2, 1), eps=0.3, kappa=0.12, csw=1.0, seed=1153, bc_t=+1, oracle=False)
    try:
        B.qcd_set_sap_domain(p.lat.ctx, (16, 6, 4, 3))
        op = CloverWilson(p.u, 0.12, 1.0, p.gammas, bc_t=+1, domain=(16, 6, 4, 3))
        op16 = copy.copy(op)
        op16.u = _half_round(op.u)
        op16.cinv = _half_round(op.cinv)
        b = p.source(2162)
        out = {}
        for shape in (0, 1):
            B.qcd_set_sap_shape(p.lat.ctx, shape)
            out[shape] = to_np(p.lat.sap(b, 2, 2, "half_gauge"))
        assert np.array_equal(out[0], out[1])
        assert rel_l2(out[0], sap.msap(op16, b, 2, 2)) <= 1e-5
    finally:
        p.close()

"""Pins of the oracle's solvers: dense LU, the free-field Fourier solution,
gauge covariance of the solution, and Algorithms 4 and 5 reaching their
tolerances (Sec. 3)."""

import numpy as np
import pytest

from lattice_inputs import gaussian_spinor, point_source, random_su3_field, random_su3_sites
from oracle import dense, solvers
from oracle.dirac import CloverWilson, dag
from oracle.gamma import gamma_chiral


def rel_resid(op, x, b):
    return np.linalg.norm((b - op.D(x)).ravel()) / np.linalg.norm(b.ravel())


def test_plain_bicgstab_matches_dense_lu():
    dims = (4, 4, 4, 4)
    g = gamma_chiral()
    u = random_su3_field(dims, 0.3, 101)
    op = CloverWilson(u, 0.12, 1.0, g)
    b = gaussian_spinor(dims, 102)
    x, it, ok = solvers.bicgstab(op.D, b, 1e-12, 1000)
    assert ok
    mat = dense.dense_D(u, op.c, op.kappa, g, -1)
    x_lu = np.linalg.solve(mat, b.ravel())
    assert np.linalg.norm(x.ravel() - x_lu) / np.linalg.norm(x_lu) < 1e-10


def free_solution(dims, kappa, b, gammas):
    """Exact D_free^-1 b by FFT with antiperiodic time (momentum p_t = (2k+1) pi / Lt)."""
    lx, ly, lz, lt = dims
    t = np.arange(lt)[:, None, None, None, None, None]
    tw = np.exp(-1j * np.pi * t / lt)
    bh = np.fft.fftn(b * tw, axes=(0, 1, 2, 3))
    kt, kz, ky, kx = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                                 indexing="ij")
    p = [2 * np.pi * kx / lx, 2 * np.pi * ky / ly, 2 * np.pi * kz / lz, (2 * kt + 1) * np.pi / lt]
    m = (1 - 2 * kappa * sum(np.cos(pm) for pm in p))[..., None, None] * np.eye(4)
    for mu in range(4):
        m = m + 2j * kappa * np.sin(p[mu])[..., None, None] * gammas[mu]
    minv = np.linalg.inv(m)
    xh = np.einsum("...st,...at->...as", minv, bh)
    return np.fft.ifftn(xh, axes=(0, 1, 2, 3)) / tw


def test_free_field_fourier_solution_8x4():
    dims = (8, 8, 8, 8)
    g = gamma_chiral()
    u = np.zeros((8, 8, 8, 8, 4, 3, 3), dtype=complex)
    u[...] = np.eye(3)
    op = CloverWilson(u, 0.12, 1.0, g, domain=(4, 4, 4, 4))
    b = gaussian_spinor(dims, 103)
    x_exact = free_solution(dims, 0.12, b, g)
    assert rel_resid(op, x_exact, b) < 1e-12
    x, _, ok = solvers.bicgstab(op.D, b, 1e-11, 2000)
    assert ok
    assert np.linalg.norm((x - x_exact).ravel()) / np.linalg.norm(x_exact.ravel()) < 1e-9
    # Algorithm 5 with SAP on A = C_inv D (C = 0 here) reaches the same solution
    xs, _, it, status = solvers.bicgstab_precdd(op, op.apply_cinv(b), 1, 2, 1e-10, 200)
    assert status == "converged"
    assert np.linalg.norm((xs - x_exact).ravel()) / np.linalg.norm(x_exact.ravel()) < 1e-8


def test_solution_gauge_covariance():
    dims = (4, 4, 4, 4)
    g = gamma_chiral()
    u = random_su3_field(dims, 0.3, 111)
    gs = random_su3_sites(dims, 112)
    ug = np.empty_like(u)
    for mu, ax in enumerate((3, 2, 1, 0)):
        ug[..., mu, :, :] = gs @ u[..., mu, :, :] @ dag(np.roll(gs, -1, axis=ax))
    op, opg = CloverWilson(u, 0.12, 1.0, g), CloverWilson(ug, 0.12, 1.0, g)
    b = gaussian_spinor(dims, 113)
    gb = np.einsum("...ab,...bs->...as", gs, b)
    x, _, _ = solvers.bicgstab(op.D, b, 1e-12, 1000)
    xg, _, _ = solvers.bicgstab(opg.D, gb, 1e-12, 1000)
    assert np.allclose(xg, np.einsum("...ab,...bs->...as", gs, x), atol=1e-9)


@pytest.mark.parametrize("n_sap,n_jac", [(1, 2), (4, 4)])
def test_algorithm5_reaches_tolerance_and_lu(n_sap, n_jac):
    dims = (4, 4, 4, 8)
    g = gamma_chiral()
    u = random_su3_field(dims, 0.3, 121)
    op = CloverWilson(u, 0.12, 1.0, g, domain=(2, 2, 2, 2))
    b = gaussian_spinor(dims, 122)
    bp = op.apply_cinv(b)
    rec = []
    x, y, it, status = solvers.bicgstab_precdd(op, bp, n_sap, n_jac, 1e-10, 200, record=rec)
    assert status == "converged"
    assert len(rec) == it
    # the recursive residual of (A M) y = b' tracks the true one
    assert np.linalg.norm((bp - op.A(x)).ravel()) / np.linalg.norm(bp.ravel()) < 1e-9
    # solving A x = C_inv b solves D x = b
    assert rel_resid(op, x, b) < 1e-8
    # SAP cuts the iteration count against the plain solver
    _, it_plain, _ = solvers.bicgstab(op.A, bp, 1e-10, 2000)
    assert it < it_plain


def test_algorithm4_defect_correction_to_1e10():
    dims = (4, 4, 4, 8)
    g = gamma_chiral()
    op = CloverWilson(random_su3_field(dims, 0.3, 131), 0.125, 1.0, g, domain=(2, 2, 2, 2))
    b = gaussian_spinor(dims, 132)
    inner = solvers.sap_inner(op, 2, 4, 1e-5, 200)
    x, outer, ok, hist = solvers.dci(op, b, 1e-10, inner)
    assert ok
    assert rel_resid(op, x, b) < 1e-10
    # each outer step gains roughly the inner tolerance (Sec. 3: O(1e-6) per step)
    assert 2 <= outer <= 4
    assert all(h1 < h0 for h0, h1 in zip(hist, hist[1:]))


def test_zero_and_point_sources():
    dims = (4, 4, 4, 4)
    op = CloverWilson(random_su3_field(dims, 0.3, 141), 0.12, 1.0, gamma_chiral(),
                      domain=(2, 2, 2, 2))
    z = np.zeros((4, 4, 4, 4, 3, 4), dtype=complex)
    x, y, it, status = solvers.bicgstab_precdd(op, z, 1, 2, 1e-10, 10)
    assert status == "converged" and it == 0 and np.abs(x).max() == 0
    b = point_source(dims, 1, 2)
    x, _, ok, _ = solvers.dci(op, b, 1e-10, solvers.sap_inner(op, 1, 2, 1e-6, 200))
    assert ok and rel_resid(op, x, b) < 1e-10


def test_maxiter_exhaustion_reports_status():
    dims = (4, 4, 4, 4)
    op = CloverWilson(random_su3_field(dims, 0.3, 151), 0.124, 1.0, gamma_chiral(),
                      domain=(2, 2, 2, 2))
    b = gaussian_spinor(dims, 152)
    _, _, it, status = solvers.bicgstab_precdd(op, op.apply_cinv(b), 0, 1, 1e-14, 2)
    assert status == "maxiter" and it == 2


def test_algorithm5_iterates_equal_textbook_bicgstab(monkeypatch):
    """Algorithm 5 is BiCGStab on the right-preconditioned operator A M_SAP
    with r~ = b and x_0 = 0 (Sec. 3).  In exact arithmetic its iterates are
    those of the independently written textbook BiCGStab on the same
    operator (r~ = r_0 = b there too), step for step: the same alpha, omega,
    x and r.  A wrong beta, omega or update in either would part them from
    the second iteration on.  After each omega step the new residual is
    orthogonal to t = (A M_SAP) s, which is what omega minimises."""
    from oracle import sap
    dims = (4, 4, 4, 8)
    g = gamma_chiral()
    op = CloverWilson(random_su3_field(dims, 0.3, 161), 0.12, 1.0, g, domain=(2, 2, 2, 2))
    b = op.apply_cinv(gaussian_spinor(dims, 162))
    n_sap, n_jac, k = 1, 2, 4
    am = lambda v: sap.am_sap(op, v, n_sap, n_jac)
    ref = []
    solvers.bicgstab(am, b, 0.0, k, record=ref)
    assert len(ref) == k

    calls = []
    orig = sap.am_sap

    def spy(op_, v, ns, nj):
        out = orig(op_, v, ns, nj)
        calls.append((v.copy(), out.copy()))
        return out

    monkeypatch.setattr(sap, "am_sap", spy)
    rec = []
    _, y, it, status = solvers.bicgstab_precdd(op, b, n_sap, n_jac, 0.0, k, record=rec)
    monkeypatch.setattr(sap, "am_sap", orig)
    assert status == "maxiter" and it == k and len(rec) == k
    bn = np.linalg.norm(b.ravel())
    for i in range(k):
        alpha, omega, rnorm2 = rec[i]
        a_ref, o_ref, x_ref, r_ref = ref[i]
        assert abs(alpha - a_ref) <= 1e-10 * abs(a_ref)
        assert abs(omega - o_ref) <= 1e-10 * abs(o_ref)
        assert abs(np.sqrt(rnorm2) - np.linalg.norm(r_ref.ravel())) <= 1e-9 * bn
        # the omega step: t = (A M) s, r_new = s - omega t, <t | r_new> = 0
        s_vec, t_vec = calls[2 * i + 1]
        r_new = s_vec - omega * t_vec
        assert abs(np.vdot(t_vec.ravel(), r_new.ravel())) <= 1e-12 * np.linalg.norm(t_vec) * bn
        assert abs(np.linalg.norm(r_new.ravel()) - np.linalg.norm(r_ref.ravel())) <= 1e-9 * bn
    # the last iterate y (before x = M_SAP y) is the textbook x
    x_ref = ref[-1][2]
    assert np.linalg.norm((y - x_ref).ravel()) <= 1e-9 * np.linalg.norm(x_ref.ravel())

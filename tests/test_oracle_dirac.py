"""Pins of the oracle's Dirac operator against closed forms, brute force and
symmetries (App. A; Sec. 3 for A = C_inv D and its domain blocks)."""

import numpy as np
import pytest

from lattice_inputs import gaussian_spinor, random_su3_field, random_su3_sites
from oracle import dense
from oracle.dirac import CloverWilson, dag, field_strength, site_mul, spin_mul
from oracle.gamma import PLANES, chiral_rotation, gamma5, gamma_chiral, gamma_paper


def free_links(dims):
    lx, ly, lz, lt = dims
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[...] = np.eye(3)
    return u


def coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    return (x, y, z, t)


@pytest.mark.parametrize("basis", ["paper", "chiral"])
@pytest.mark.parametrize("bc_t", [-1, 1])
def test_free_field_plane_wave(basis, bc_t):
    """U = 1: D e^{ipn} u = [1 - 2 kappa sum cos p + 2 i kappa sum gamma sin p] e^{ipn} u,
    with p_t = (2 n_t + 1) pi / Lt for antiperiodic time; the clover vanishes."""
    g = gamma_paper() if basis == "paper" else gamma_chiral()
    dims = (4, 6, 4, 8)
    kappa = 0.13
    op = CloverWilson(free_links(dims), kappa, 1.7, g, bc_t=bc_t)
    assert np.abs(op.c).max() < 1e-15
    rng = np.random.default_rng(7)
    for nk in [(1, 2, 3, 1), (0, 5, 1, 6), (3, 0, 2, 3)]:
        p = [2 * np.pi * nk[mu] / dims[mu] for mu in range(3)]
        shift = 1 if bc_t == -1 else 0
        p.append((2 * nk[3] + shift) * np.pi / dims[3])
        phase = np.exp(1j * sum(p[mu] * coords(dims)[mu] for mu in range(4)))
        u_col = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
        psi = phase[..., None, None] * u_col
        m = (1 - 2 * kappa * sum(np.cos(p))) * np.eye(4)
        m = m + 2j * kappa * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[..., None, None] * np.einsum("st,at->as", m, u_col)
        assert np.allclose(op.D(psi), expect, atol=1e-12)


@pytest.mark.parametrize("basis", ["paper", "chiral"])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_dense_brute_force_matches_stencil(basis, dims):
    g = gamma_paper() if basis == "paper" else gamma_chiral()
    u = random_su3_field(dims, 0.4, 11)
    op = CloverWilson(u, 0.12, 1.3, g, bc_t=-1)
    mat = dense.dense_D(u, op.c, op.kappa, g, -1)
    x = gaussian_spinor(dims, 12)
    assert np.allclose(op.D(x).ravel(), mat @ x.ravel(), atol=1e-12)
    # D^dag = gamma_5 D gamma_5 against the conjugate transpose of the dense D
    assert np.allclose(op.Ddag(x).ravel(), mat.conj().T @ x.ravel(), atol=1e-12)
    # A = C_inv D
    assert np.allclose(op.A(x), op.apply_cinv(op.D(x)), atol=1e-12)


def test_gamma5_hermiticity_random_vectors():
    dims = (4, 4, 4, 4)
    g = gamma_chiral()
    op = CloverWilson(random_su3_field(dims, 0.3, 21), 0.12, 1.0, g)
    x = gaussian_spinor(dims, 22)
    y = gaussian_spinor(dims, 23)
    lhs = np.vdot(y.ravel(), op.D(x).ravel())
    rhs = np.vdot(op.Ddag(y).ravel(), x.ravel())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def gauge_transform(u, gsite, bc_dims):
    """U^g_mu(n) = g(n) U_mu(n) g(n + mu)^dag."""
    out = np.empty_like(u)
    axis = (3, 2, 1, 0)
    for mu in range(4):
        gf = np.roll(gsite, -1, axis=axis[mu])
        out[..., mu, :, :] = gsite @ u[..., mu, :, :] @ dag(gf)
    return out


@pytest.mark.parametrize("basis", ["paper", "chiral"])
def test_gauge_covariance(basis):
    """D[U^g] (g x) = g (D[U] x), clover included; F -> g F g^dag."""
    g = gamma_paper() if basis == "paper" else gamma_chiral()
    dims = (4, 4, 2, 6)
    u = random_su3_field(dims, 0.5, 31)
    gs = random_su3_sites(dims, 32)
    ug = gauge_transform(u, gs, dims)
    op = CloverWilson(u, 0.11, 1.2, g)
    opg = CloverWilson(ug, 0.11, 1.2, g)
    x = gaussian_spinor(dims, 33)
    gx = np.einsum("...ab,...bs->...as", gs, x)
    lhs = opg.D(gx)
    rhs = np.einsum("...ab,...bs->...as", gs, op.D(x))
    assert np.allclose(lhs, rhs, atol=1e-12)
    f = field_strength(u)
    fg = field_strength(ug)
    assert np.allclose(fg, gs[..., None, :, :] @ f @ dag(gs)[..., None, :, :], atol=1e-12)


def test_pure_gauge_has_no_field_strength_and_free_spectrum():
    dims = (4, 4, 4, 4)
    gs = random_su3_sites(dims, 41)
    ug = gauge_transform(free_links(dims), gs, dims)
    assert np.abs(field_strength(ug)).max() < 1e-13


def test_basis_equivalence():
    """D in the chiral basis equals S D_paper S^dag on the spin index."""
    dims = (4, 4, 4, 4)
    u = random_su3_field(dims, 0.3, 51)
    opp = CloverWilson(u, 0.125, 1.0, gamma_paper())
    opc = CloverWilson(u, 0.125, 1.0, gamma_chiral())
    s = chiral_rotation()
    x = gaussian_spinor(dims, 52)
    lhs = opc.D(x)
    rhs = spin_mul(s, opp.D(spin_mul(s.conj().T, x)))
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_clover_algebra():
    dims = (4, 4, 4, 4)
    g = gamma_chiral()
    op = CloverWilson(random_su3_field(dims, 0.4, 61), 0.12, 1.1, g)
    c = op.c
    assert np.allclose(c, dag(c), atol=1e-14)
    g5 = np.kron(np.eye(3), gamma5(g))
    assert np.allclose(c @ g5, g5 @ c, atol=1e-14)
    assert np.allclose((np.eye(12) + c) @ op.cinv, np.eye(12), atol=1e-13)
    f = field_strength(op.u)
    assert np.allclose(f, -dag(f), atol=1e-14)


@pytest.mark.parametrize("basis", ["paper", "chiral"])
def test_constant_abelian_field_closed_form(basis):
    """U_1(n) = exp(i B n_2 T), U_2 = exp(-i B L_2 n_1 T) on the n_2 = L_2 - 1
    slice, identity elsewhere: every 1-2 plaquette equals exp(-i B T), so
    F_hat_12 = -i sin(B T), the other planes vanish, and
    C = kappa c_SW sigma_12 (x) sin(B T) on every site."""
    g = gamma_paper() if basis == "paper" else gamma_chiral()
    dims = (4, 6, 2, 2)
    lx, ly, lz, lt = dims
    k = 1
    bmag = 2 * np.pi * k / (lx * ly)
    tdiag = np.array([1.0, -1.0, 0.0])
    x, y, z, t = coords(dims)
    u = free_links(dims)
    u[..., 0, :, :] = np.einsum("...a,ab->...ab", np.exp(1j * bmag * y[..., None] * tdiag), np.eye(3))
    ph2 = np.exp(-1j * bmag * ly * x[..., None] * tdiag)
    edge = (y == ly - 1)
    u2 = np.einsum("...a,ab->...ab", ph2, np.eye(3))
    u[..., 1, :, :] = np.where(edge[..., None, None], u2, np.eye(3))
    kappa, csw = 0.12, 1.4
    op = CloverWilson(u, kappa, csw, g)
    f = field_strength(u)
    expect12 = -1j * np.diag(np.sin(bmag * tdiag))
    assert np.allclose(f[..., 0, :, :], expect12, atol=1e-14)
    assert np.abs(f[..., 1:, :, :]).max() < 1e-14
    # sigma_12 = i g1 g2 = diag(-1, 1, -1, 1), written out by hand (equal in both bases)
    sigma12 = np.diag([-1.0, 1.0, -1.0, 1.0])
    c_expect = kappa * csw * np.kron(np.diag(np.sin(bmag * tdiag)), sigma12)
    assert np.allclose(op.c, c_expect, atol=1e-14)


def test_domain_partition_identity_and_support():
    dims = (4, 4, 4, 8)
    op = CloverWilson(random_su3_field(dims, 0.3, 71), 0.12, 1.0, gamma_chiral(),
                      domain=(2, 2, 2, 2))
    x = gaussian_spinor(dims, 72)
    total = sum(op.A_block(x, r, c) for r in (0, 1) for c in (0, 1))
    assert np.allclose(total, op.A(x), atol=1e-13)
    # A_EE maps a vector supported on one domain into that domain
    mask = np.zeros(x.shape[:4])
    mask[0:2, 0:2, 0:2, 0:2] = 1.0        # domain (0,0,0,0): even
    xd = x * mask[..., None, None]
    y = op.A_block(xd, 0, 0)
    assert np.abs(y * (1 - mask)[..., None, None]).max() == 0
    # and A_OE of it only reaches odd sites adjacent to the domain surface
    z = op.A_block(xd, 1, 0)
    assert np.abs(z * op.mask(0)).max() == 0


def test_paper_form_of_A():
    """A x = x - kappa sum_mu [C_inv T+ x(n+mu) + C_inv T- x(n-mu)] (Sec. 3)."""
    dims = (2, 2, 4, 4)
    g = gamma_paper()
    u = random_su3_field(dims, 0.3, 81)
    op = CloverWilson(u, 0.12, 1.0, g)
    mat_d = dense.dense_D(u, op.c, op.kappa, g, -1)
    v = 12 * np.prod(dims)
    cinv_blk = np.zeros((v, v), dtype=complex)
    cinv = op.cinv.reshape(-1, 12, 12)
    for i in range(cinv.shape[0]):
        cinv_blk[12 * i:12 * i + 12, 12 * i:12 * i + 12] = cinv[i]
    x = gaussian_spinor(dims, 82)
    assert np.allclose(op.A(x).ravel(), cinv_blk @ mat_d @ x.ravel(), atol=1e-12)


def test_pointwise_matches_whole_lattice():
    """The site-by-site form used for sampled checks of large lattices equals
    the whole-lattice operator."""
    from oracle import pointwise
    dims = (4, 4, 2, 6)
    for basis, g in (("paper", gamma_paper()), ("chiral", gamma_chiral())):
        u = random_su3_field(dims, 0.5, 91)
        op = CloverWilson(u, 0.13, 1.2, g, bc_t=-1)
        x = gaussian_spinor(dims, 92)
        full = op.D(x)
        rng = np.random.default_rng(3)
        for _ in range(12):
            c = tuple(int(rng.integers(0, dims[mu])) for mu in range(4))
            got = pointwise.D_at(u, x, c, 0.13, 1.2, g, -1)
            assert np.allclose(got, full[c[3], c[2], c[1], c[0]], atol=1e-12)


def test_fast_generator_matches_reference_generator():
    """The torch-exponentiated generator draws the same links as the numpy one."""
    from lattice_inputs import random_su3_field_fast
    a = random_su3_field((4, 4, 4, 8), 0.3, 7)
    b = random_su3_field_fast((4, 4, 4, 8), 0.3, 7, device="cpu", chunk=1000)
    assert np.abs(a - b).max() < 1e-13

"""Pins of Algorithms 1-3 against the polynomials of Sec. 3 built from dense
blocks of A (brute-force dense D, block-diagonal C_inv)."""

import numpy as np
import pytest

from lattice_inputs import gaussian_spinor, random_su3_field
from oracle import dense, sap
from oracle.dirac import CloverWilson
from oracle.gamma import gamma_chiral


def setup(dims, domain, seed=91, kappa=0.12, csw=1.0):
    g = gamma_chiral()
    u = random_su3_field(dims, 0.3, seed)
    op = CloverWilson(u, kappa, csw, g, domain=domain)
    mat_d = dense.dense_D(u, op.c, op.kappa, g, -1)
    v = 12 * int(np.prod(dims))
    cinv = op.cinv.reshape(-1, 12, 12)
    cb = np.zeros((v, v), dtype=complex)
    for i in range(cinv.shape[0]):
        cb[12 * i:12 * i + 12, 12 * i:12 * i + 12] = cinv[i]
    a = cb @ mat_d
    col = np.repeat(dense.colour_of_sites(dims, domain), 12)
    dom = np.repeat(dense.domain_of_sites(dims, domain), 12)
    return op, a, col, dom


def blocks(a, col):
    e = np.where(col == 0)[0]
    o = np.where(col == 1)[0]
    return e, o, a[np.ix_(e, e)], a[np.ix_(e, o)], a[np.ix_(o, e)], a[np.ix_(o, o)]


def neumann(a_cc, v, n_jac):
    """sum_{j=0}^{n_jac} (I - A_cc)^j v by dense matrix-vector products."""
    term = v.copy()
    acc = v.copy()
    for _ in range(n_jac):
        term = term - a_cc @ term
        acc = acc + term
    return acc


DIMS, DOMAIN = (4, 4, 4, 4), (2, 2, 2, 2)


@pytest.fixture(scope="module")
def lat():
    return setup(DIMS, DOMAIN)


def test_domain_blocks_are_block_diagonal(lat):
    op, a, col, dom = lat
    e, o, aee, aeo, aoe, aoo = blocks(a, col)
    same = dom[e][:, None] == dom[e][None, :]
    assert np.abs(aee[~same]).max() == 0
    # the oracle's block operators equal the dense blocks
    x = gaussian_spinor(DIMS, 92)
    xv = x.ravel()
    for r, c, m, ri, ci in [(0, 0, aee, e, e), (0, 1, aeo, e, o), (1, 0, aoe, o, e), (1, 1, aoo, o, o)]:
        y = op.A_block(x, r, c).ravel()
        assert np.allclose(y[ri], m @ xv[ci], atol=1e-12)
        other = o if r == 0 else e
        assert np.abs(y[other]).max() == 0


@pytest.mark.parametrize("n_jac", [1, 2, 4])
def test_jacobi_is_truncated_neumann_series(lat, n_jac):
    op, a, col, _ = lat
    e, o, aee, _, _, aoo = blocks(a, col)
    b = gaussian_spinor(DIMS, 93)
    for c, idx, acc in [(0, e, aee), (1, o, aoo)]:
        x = sap.jacobi(op, b, c, n_jac).ravel()
        assert np.allclose(x[idx], neumann(acc, b.ravel()[idx], n_jac), atol=1e-12)


def dense_k(v, e, o, aoe, inv_e, inv_o):
    ye = inv_e(v[e])
    yo = inv_o(v[o] - aoe @ ye)
    out = np.zeros_like(v)
    out[e] = ye
    out[o] = yo
    return out


@pytest.mark.parametrize("n_sap,n_jac", [(0, 1), (1, 2), (4, 4)])
def test_msap_is_eq_msap_polynomial(lat, n_sap, n_jac):
    """Algorithm 1 == K sum_{j=0}^{n_sap} (1 - A K)^j with K from dense blocks."""
    op, a, col, _ = lat
    e, o, aee, _, aoe, aoo = blocks(a, col)
    k = lambda v: dense_k(v, e, o, aoe, lambda w: neumann(aee, w, n_jac),
                          lambda w: neumann(aoo, w, n_jac))
    b = gaussian_spinor(DIMS, 94)
    v = b.ravel().copy()
    acc = np.zeros_like(v)
    for _ in range(n_sap + 1):
        acc += v
        v = v - a @ k(v)
    expect = k(acc)
    got = sap.msap(op, b, n_sap, n_jac).ravel()
    assert np.allclose(got, expect, atol=1e-11)
    # A M_SAP = I - (I - A K)^{n_sap + 1}
    am = sap.am_sap(op, b, n_sap, n_jac).ravel()
    assert np.allclose(am, b.ravel() - v, atol=1e-11)


def test_exact_block_inverse_makes_ak_upper_triangular(lat):
    """With B = A_cc^-1 the odd-odd block of A K is I and the odd-even block is 0."""
    op, a, col, _ = lat
    e, o, aee, aeo, aoe, aoo = blocks(a, col)
    iee, ioo = np.linalg.inv(aee), np.linalg.inv(aoo)
    n = a.shape[0]
    kmat = np.zeros((n, n), dtype=complex)
    kmat[np.ix_(e, e)] = iee
    kmat[np.ix_(o, o)] = ioo
    kmat[np.ix_(o, e)] = -ioo @ aoe @ iee
    ak = a @ kmat
    assert np.allclose(ak[np.ix_(o, o)], np.eye(len(o)), atol=1e-11)
    assert np.abs(ak[np.ix_(o, e)]).max() < 1e-11
    assert np.allclose(ak[np.ix_(e, o)], aeo @ ioo, atol=1e-11)
    # the oracle's K with exact inverses agrees with the dense K
    b = gaussian_spinor(DIMS, 95)
    exact = lambda v, c: _exact(op, a, col, v, c)
    assert np.allclose(sap.k_apply(op, b, 1, exact=exact).ravel(), kmat @ b.ravel(), atol=1e-11)


def _exact(op, a, col, v, c):
    idx = np.where(col == c)[0]
    out = np.zeros(v.size, dtype=complex)
    out[idx] = np.linalg.solve(a[np.ix_(idx, idx)], v.ravel()[idx])
    return out.reshape(v.shape)


def test_msap_series_closed_form_helper(lat):
    op, _, _, _ = lat
    b = gaussian_spinor(DIMS, 96)
    assert np.allclose(sap.msap(op, b, 2, 3), sap.msap_series(op, b, 2, 3), atol=1e-11)


def test_single_site_domains_degenerate_case():
    """1^4 domains: A_EE = I (no intra-domain hops), so B_EE = I and SAP is
    red/black Gauss-Seidel on sites."""
    dims = (2, 2, 2, 2)
    op, a, col, _ = setup(dims, (1, 1, 1, 1), seed=97)
    e, o, aee, _, _, aoo = blocks(a, col)
    assert np.allclose(aee, np.eye(len(e)))
    b = gaussian_spinor(dims, 98)
    assert np.allclose(sap.jacobi(op, b, 0, 3), op.mask(0) * b, atol=1e-14)

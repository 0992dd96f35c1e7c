"""Pins of the oracle gradients of L = Re(eta^dag D^-1 b): dense LU closed form
for d/db and central finite differences along random su(3) directions for
d/dU, hopping and clover parts separately."""

import numpy as np
import pytest

from lattice_inputs import gaussian_spinor, random_su3_algebra, random_su3_field
from oracle import dense, grad
from oracle.dirac import CloverWilson
from oracle.gamma import gamma5, gamma_chiral


def loss_lu(u, kappa, csw, g, eta, b):
    op = CloverWilson(u, kappa, csw, g)
    mat = dense.dense_D(u, op.c, kappa, g, -1)
    x = np.linalg.solve(mat, b.ravel())
    return float(np.vdot(eta.ravel(), x).real)


def test_grad_b_closed_form():
    dims = (2, 2, 4, 4)
    g = gamma_chiral()
    u = random_su3_field(dims, 0.3, 161)
    op = CloverWilson(u, 0.12, 1.0, g)
    eta, b = gaussian_spinor(dims, 162), gaussian_spinor(dims, 163)
    lam, _ = grad.gradients(op, eta, b)
    mat = dense.dense_D(u, op.c, op.kappa, g, -1)
    lam_lu = np.linalg.solve(mat.conj().T, eta.ravel())
    assert np.allclose(lam.ravel(), lam_lu, atol=1e-10)
    # gamma_5 D^-1 gamma_5 form of D^-dag
    g5 = np.kron(np.eye(np.prod(dims) * 3), gamma5(g))
    assert np.allclose(g5 @ np.linalg.solve(mat, g5 @ eta.ravel()), lam_lu, atol=1e-10)
    # central finite difference in a random direction of b
    d = gaussian_spinor(dims, 164)
    h = 1e-4
    fd = (loss_lu(u, 0.12, 1.0, g, eta, b + h * d) - loss_lu(u, 0.12, 1.0, g, eta, b - h * d)) / (2 * h)
    assert abs(fd - np.vdot(lam.ravel(), d.ravel()).real) < 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("csw", [0.0, 1.3])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_grad_u_finite_difference(dims, csw):
    g = gamma_chiral()
    kappa = 0.12
    u = random_su3_field(dims, 0.3, 171)
    op = CloverWilson(u, kappa, csw, g)
    eta, b = gaussian_spinor(dims, 172), gaussian_spinor(dims, 173)
    _, graw = grad.gradients(op, eta, b)
    pi = grad.project_su3(graw, u)
    x_dir = random_su3_algebra(u.shape[:-2], 174)
    h = 1e-4
    e_plus = _expm_stack(h * x_dir) @ u
    e_minus = _expm_stack(-h * x_dir) @ u
    fd = (loss_lu(e_plus, kappa, csw, g, eta, b) - loss_lu(e_minus, kappa, csw, g, eta, b)) / (2 * h)
    analytic = np.sum(np.conj(pi) * x_dir).real
    raw = np.sum(np.conj(graw) * (x_dir @ u)).real
    assert abs(raw - analytic) < 1e-10 * max(1.0, abs(analytic))
    assert abs(fd - analytic) < 1e-6 * max(1.0, abs(analytic))


def _expm_stack(m):
    w, v = np.linalg.eigh(-1j * m)          # -i m is Hermitian for anti-Hermitian m
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), v.conj())


def test_projection_is_traceless_antihermitian():
    m = np.random.default_rng(5).standard_normal((10, 3, 3)) * (1 + 1j)
    t = grad.traceless_antihermitian(m)
    assert np.allclose(t, -np.swapaxes(t, -1, -2).conj())
    assert np.allclose(np.trace(t, axis1=-2, axis2=-1), 0)


@pytest.mark.slow
def test_grad_u_finite_difference_8x4():
    """Central difference at 8^4 with iterative float64 solves."""
    dims = (8, 8, 8, 8)
    g = gamma_chiral()
    kappa, csw = 0.12, 1.0
    u = random_su3_field(dims, 0.3, 181)
    op = CloverWilson(u, kappa, csw, g)
    eta, b = gaussian_spinor(dims, 182), gaussian_spinor(dims, 183)
    _, graw = grad.gradients(op, eta, b, tol=1e-13)
    pi = grad.project_su3(graw, u)
    x_dir = random_su3_algebra(u.shape[:-2], 184)
    h = 1e-4
    lp = grad.loss(CloverWilson(_expm_stack(h * x_dir) @ u, kappa, csw, g), eta, b)
    lm = grad.loss(CloverWilson(_expm_stack(-h * x_dir) @ u, kappa, csw, g), eta, b)
    fd = (lp - lm) / (2 * h)
    analytic = np.sum(np.conj(pi) * x_dir).real
    assert abs(fd - analytic) < 1e-6 * max(1.0, abs(analytic))

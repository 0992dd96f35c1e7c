"""Pins of the gamma algebra (App. A) in both bases."""

import numpy as np
import pytest

from oracle.gamma import PLANES, chiral_rotation, gamma5, gamma_chiral, gamma_paper, sigma


@pytest.mark.parametrize("basis", [gamma_paper, gamma_chiral])
def test_clifford_and_hermiticity(basis):
    g = basis()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))


@pytest.mark.parametrize("basis", [gamma_paper, gamma_chiral])
def test_gamma5_properties(basis):
    g = basis()
    g5 = gamma5(g)
    assert np.allclose(g5, g5.conj().T)
    assert np.allclose(g5 @ g5, np.eye(4))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu], -g[mu] @ g5)
    for mu, nu in PLANES:
        s = sigma(g, mu, nu)
        assert np.allclose(s, s.conj().T)
        assert np.allclose(s @ g5, g5 @ s)


def test_paper_matrices_as_printed():
    g = gamma_paper()
    # gamma_4 is the diagonal one in App. A
    assert np.allclose(g[3], np.diag([1, 1, -1, -1]))
    assert g[0][0, 3] == 1j and g[0][3, 0] == -1j
    assert g[1][1, 2] == -1 and g[1][3, 0] == 1
    assert g[2][0, 2] == 1j and g[2][1, 3] == -1j


def test_chiral_basis_form():
    s = chiral_rotation()
    assert np.allclose(s @ s.conj().T, np.eye(4))
    g = gamma_chiral()
    assert np.allclose(gamma5(g), np.diag([1, 1, -1, -1]))
    z = np.zeros((2, 2))
    i2 = np.eye(2)
    assert np.allclose(g[3], np.block([[z, i2], [i2, z]]))
    pauli = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
    for k in range(3):
        expect = np.block([[z, -1j * pauli[k]], [1j * pauli[k], z]])
        assert np.allclose(g[k], expect)


def test_sigma_squares_to_one():
    """sigma_{mu nu}^2 = 1 for mu != nu: with anticommuting gammas,
    [g_mu, g_nu] = 2 g_mu g_nu and (i g_mu g_nu)^2 = -g_mu g_nu g_mu g_nu = 1.
    This fixes the factor i/2 of App. A (a factor 1 would give 4)."""
    for basis in (gamma_paper, gamma_chiral):
        g = basis()
        for mu, nu in PLANES:
            s = sigma(g, mu, nu)
            assert np.allclose(s @ s, np.eye(4), atol=1e-15)


def test_sigma_hand_written_entries():
    """sigma_12 = i g1 g2 and sigma_34 = i g3 g4 multiplied out by hand from
    the printed App. A matrices: g1 g2 = diag(i, -i, i, -i), so
    sigma_12 = diag(-1, 1, -1, 1) (the same in the chiral basis, which
    rotates the two equal 2x2 blocks onto each other); sigma_34 couples the
    upper and lower spin pairs through diag(1, -1), and becomes
    diag(1, -1, -1, 1) in the chiral basis."""
    s12 = np.diag([-1.0, 1.0, -1.0, 1.0])
    s34_paper = np.array([[0, 0, 1, 0], [0, 0, 0, -1], [1, 0, 0, 0], [0, -1, 0, 0]], dtype=float)
    s34_chiral = np.diag([1.0, -1.0, -1.0, 1.0])
    assert np.allclose(sigma(gamma_paper(), 0, 1), s12, atol=1e-15)
    assert np.allclose(sigma(gamma_chiral(), 0, 1), s12, atol=1e-15)
    assert np.allclose(sigma(gamma_paper(), 2, 3), s34_paper, atol=1e-15)
    assert np.allclose(sigma(gamma_chiral(), 2, 3), s34_chiral, atol=1e-15)

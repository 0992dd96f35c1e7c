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

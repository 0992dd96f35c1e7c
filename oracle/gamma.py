"""Gamma matrices (App. A) and the chiral rotation.

The paper prints gamma_1..gamma_4 in a basis where gamma_4 is diagonal and
notes that any unitarily equivalent representation may be used.  The CUDA
path works in the chiral basis gamma'_mu = S gamma_mu S^dag, with
S = (1/sqrt 2) [[1, 1], [1, -1]] acting on the (upper, lower) spin pairs,
where gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 becomes diag(1, 1, -1, -1).
"""

import numpy as np


def gamma_paper():
    """gamma_1..gamma_4 exactly as printed in App. A; shape (4, 4, 4)."""
    i = 1j
    g1 = np.array([[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]])
    g2 = np.array([[0, 0, 0, 1], [0, 0, -1, 0], [0, -1, 0, 0], [1, 0, 0, 0]])
    g3 = np.array([[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]])
    g4 = np.diag([1, 1, -1, -1])
    return np.array([g1, g2, g3, g4], dtype=np.complex128)


def chiral_rotation():
    """The unitary S taking the paper basis to the chiral basis."""
    i2 = np.eye(2)
    return np.block([[i2, i2], [i2, -i2]]).astype(np.complex128) / np.sqrt(2.0)


def gamma_chiral():
    """gamma'_mu = S gamma_mu S^dag for the four directions; shape (4, 4, 4)."""
    s = chiral_rotation()
    return np.array([s @ g @ s.conj().T for g in gamma_paper()])


def gammas_for(basis):
    if basis == "chiral":
        return gamma_chiral()
    if basis == "paper":
        return gamma_paper()
    raise ValueError(f"unknown gamma basis {basis!r}")


def gamma5(gammas):
    """gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 (the paper leaves it undefined)."""
    return gammas[0] @ gammas[1] @ gammas[2] @ gammas[3]


def sigma(gammas, mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] (App. A)."""
    g = gammas
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


PLANES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))

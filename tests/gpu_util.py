"""Shared set-up for the GPU parity tests: one seeded problem, handed to both
the CUDA library (through the C ABI) and the float64 oracle."""

import numpy as np

from lattice_inputs import gaussian_spinor, random_su3_field
from oracle.dirac import CloverWilson
from oracle.gamma import gamma_chiral, gamma_paper


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


class Problem:
    """A gauge field, parameters and the two implementations of D on it."""

    def __init__(self, dims, domain=(4, 4, 4, 4), eps=0.3, kappa=0.12, csw=1.0, seed=1001, bc_t=-1,
                 basis="chiral", oracle=True):
        from paper_2109_10687_gb300.lattice import Lattice
        self.dims, self.domain = tuple(dims), tuple(domain)
        self.kappa, self.csw, self.bc_t, self.basis = kappa, csw, bc_t, basis
        self.u = random_su3_field(dims, eps, seed)
        self.lat = Lattice(dims, domain, bc_t, basis).setup(self.u, kappa, csw)
        g = gamma_chiral() if basis == "chiral" else gamma_paper()
        self.gammas = g
        self.op = CloverWilson(self.u, kappa, csw, g, bc_t=bc_t, domain=domain) if oracle else None

    def source(self, seed, nrhs=None):
        return gaussian_spinor(self.dims, seed, nrhs)

    def close(self):
        self.lat.close()

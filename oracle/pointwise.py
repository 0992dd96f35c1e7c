"""Site-by-site evaluation of D x (App. A) for sampled sites of large lattices.

The whole-lattice oracle in ``dirac`` keeps a dense 12x12 clover matrix per
site, which does not fit for 32^4 and larger lattices.  These functions take
the same definitions one site at a time -- the links around the site, the
four-leaf field strength at the site, the eight hops -- so that parity tests
can check any sampled output of a full-size GPU application.
"""

import numpy as np

from .gamma import PLANES, sigma


def _wrap(dims, c):
    return tuple(int(c[mu]) % dims[mu] for mu in range(4))


def link(u, dims, c, mu):
    """U_mu at coordinates c = (x, y, z, t), periodic."""
    x, y, z, t = _wrap(dims, c)
    return u[t, z, y, x, mu]


def spinor(psi, dims, c):
    x, y, z, t = _wrap(dims, c)
    return psi[t, z, y, x]


def _shift(c, mu, k):
    c = list(c)
    c[mu] += k
    return c


def field_strength_at(u, dims, c, mu, nu):
    """F_hat_{mu nu}(c) = (Q - Q^dag) / 8 from the four leaves through c."""
    def L(d, dm, dn):
        cc = _shift(_shift(c, mu, dm), nu, dn)
        return link(u, dims, cc, d)

    h = lambda m: m.conj().T
    q = (L(mu, 0, 0) @ L(nu, 1, 0) @ h(L(mu, 0, 1)) @ h(L(nu, 0, 0))
         + L(nu, 0, 0) @ h(L(mu, -1, 1)) @ h(L(nu, -1, 0)) @ L(mu, -1, 0)
         + h(L(mu, -1, 0)) @ h(L(nu, -1, -1)) @ L(mu, -1, -1) @ L(nu, 0, -1)
         + h(L(nu, 0, -1)) @ L(mu, 0, -1) @ L(nu, 1, -1) @ h(L(mu, 0, 0)))
    return (q - h(q)) / 8.0


def clover_at(u, dims, c, kappa, csw, gammas):
    """12x12 clover matrix C at site c (index 4 colour + spin)."""
    out = np.zeros((12, 12), dtype=np.complex128)
    for mu, nu in PLANES:
        out += np.kron(field_strength_at(u, dims, c, mu, nu), sigma(gammas, mu, nu))
    return 1j * kappa * csw * out


def D_at(u, psi, c, kappa, csw, gammas, bc_t):
    """(D psi) at site c = (x, y, z, t), shape (3, 4)."""
    lt, lz, ly, lx = u.shape[:4]
    dims = (lx, ly, lz, lt)
    eye = np.eye(4)
    v = spinor(psi, dims, c)
    out = v + (clover_at(u, dims, c, kappa, csw, gammas) @ v.reshape(12)).reshape(3, 4)
    hop = np.zeros((3, 4), dtype=np.complex128)
    for mu in range(4):
        cf = _shift(c, mu, 1)
        sf = bc_t if (mu == 3 and cf[3] == dims[3]) else 1.0
        hop += sf * (link(u, dims, c, mu) @ spinor(psi, dims, cf)) @ (eye - gammas[mu]).T
        cb = _shift(c, mu, -1)
        sb = bc_t if (mu == 3 and cb[3] < 0) else 1.0
        hop += sb * (link(u, dims, cb, mu).conj().T @ spinor(psi, dims, cb)) @ (eye + gammas[mu]).T
    return out - kappa * hop

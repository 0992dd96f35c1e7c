"""Clover-Wilson Dirac operator, float64, whole-lattice numpy (App. A, Sec. 3).

Conventions (the readings are listed with their reasons in the design notes):

* fields use the canonical layout of ``lattice_inputs``: a quark field is
  ``[t][z][y][x][colour 3][spin 4]``; links are ``[t][z][y][x][mu][3][3]``;
* the hop in direction +mu couples x(n + mu) through U_mu(n), the hop in -mu
  couples x(n - mu) through U_{-mu}(n) = U_mu(n - mu)^dag (the form of the
  stencil in Sec. 3 and App. A);
* space is periodic; time is periodic (bc_t = +1) or antiperiodic
  (bc_t = -1), the sign multiplying every hop that crosses t = Lt-1 <-> 0;
  the sign is applied to the hop, never to a link (the clover leaves use the
  links without it);
* a 12x12 site matrix acts on the index (colour a, spin alpha) -> 4 a + alpha.
"""

import numpy as np

from .gamma import PLANES, gamma5, sigma

# numpy axis of the [t][z][y][x] site block for direction mu = x, y, z, t
AXIS = (3, 2, 1, 0)


def site_dims(field):
    """(Lx, Ly, Lz, Lt) of a field in canonical layout."""
    lt, lz, ly, lx = field.shape[:4]
    return (lx, ly, lz, lt)


def shift_fwd(f, mu, bc_t):
    """g(n) = f(n + mu), times bc_t where the hop crosses the time boundary."""
    g = np.roll(f, -1, axis=AXIS[mu])
    if mu == 3 and bc_t != 1:
        g[-1] *= bc_t
    return g


def shift_bwd(f, mu, bc_t):
    """g(n) = f(n - mu), times bc_t where the hop crosses the time boundary."""
    g = np.roll(f, 1, axis=AXIS[mu])
    if mu == 3 and bc_t != 1:
        g[0] *= bc_t
    return g


def link_at(u_mu, shifts):
    """U(n + sum_k s_k e_k) for a single-direction link field ``[t][z][y][x][3][3]``.

    ``shifts`` is a dict {direction: integer offset}.
    """
    out = u_mu
    for d, s in shifts.items():
        if s:
            out = np.roll(out, -s, axis=AXIS[d])
    return out


def dag(m):
    return np.swapaxes(m, -1, -2).conj()


def colour_mul(m, psi):
    """(M psi)_{a s} = sum_b M_{ab} psi_{b s} per site."""
    return np.einsum("...ab,...bs->...as", m, psi)


def spin_mul(p, psi):
    """(P psi)_{a s} = sum_t P_{st} psi_{a t} with one 4x4 spin matrix."""
    return np.einsum("st,...at->...as", p, psi)


def site_mul(m12, psi):
    """Apply a 12x12 site matrix to a quark field."""
    v = psi.reshape(psi.shape[:-2] + (12,))
    return np.einsum("...ij,...j->...i", m12, v).reshape(psi.shape)


def hop(u, x, gammas, bc_t, fwd_mask=None, bwd_mask=None):
    """H x = sum_mu [(1 - g_mu) U_mu(n) x(n+mu) + (1 + g_mu) U_mu(n-mu)^dag x(n-mu)].

    ``fwd_mask[mu]`` / ``bwd_mask[mu]`` (0/1 site arrays) keep only a subset of
    the hops, selected by the site n the result lands on.
    """
    eye = np.eye(4)
    out = np.zeros_like(x)
    for mu in range(4):
        umu = u[..., mu, :, :]
        fwd = spin_mul(eye - gammas[mu], colour_mul(umu, shift_fwd(x, mu, bc_t)))
        ub = dag(link_at(umu, {mu: -1}))
        bwd = spin_mul(eye + gammas[mu], colour_mul(ub, shift_bwd(x, mu, bc_t)))
        if fwd_mask is not None:
            fwd = fwd * fwd_mask[mu][..., None, None]
            bwd = bwd * bwd_mask[mu][..., None, None]
        out += fwd + bwd
    return out


def clover_leaves(u, mu, nu):
    """Q_{mu nu}(n): the four plaquettes in the mu-nu plane through n, all
    oriented the same way (the standard four-leaf clover; App. A names
    F_{mu nu} without giving its form)."""
    um = u[..., mu, :, :]
    un = u[..., nu, :, :]
    q1 = (um @ link_at(un, {mu: 1}) @ dag(link_at(um, {nu: 1})) @ dag(un))
    q2 = (un @ dag(link_at(um, {mu: -1, nu: 1})) @ dag(link_at(un, {mu: -1}))
          @ link_at(um, {mu: -1}))
    q3 = (dag(link_at(um, {mu: -1})) @ dag(link_at(un, {mu: -1, nu: -1}))
          @ link_at(um, {mu: -1, nu: -1}) @ link_at(un, {nu: -1}))
    q4 = (dag(link_at(un, {nu: -1})) @ link_at(um, {nu: -1})
          @ link_at(un, {mu: 1, nu: -1}) @ dag(um))
    return q1 + q2 + q3 + q4


def field_strength(u):
    """F_hat_{mu nu} = (Q - Q^dag) / 8 for the six planes mu < nu, anti-Hermitian.

    Returns ``[t][z][y][x][plane 6][3][3]`` in the plane order of ``PLANES``.
    """
    out = []
    for mu, nu in PLANES:
        q = clover_leaves(u, mu, nu)
        out.append((q - dag(q)) / 8.0)
    return np.stack(out, axis=-3)


def clover_term(u, kappa, csw, gammas):
    """C = (i/2) kappa c_SW sum_{mu,nu} sigma_{mu nu} F_{mu nu}
         = i kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) F_hat_{mu nu}   (App. A).

    Returned as a 12x12 Hermitian matrix per site.
    """
    f = field_strength(u)
    c = np.zeros(f.shape[:4] + (3, 4, 3, 4), dtype=np.complex128)
    for p, (mu, nu) in enumerate(PLANES):
        c += np.einsum("...ab,st->...asbt", f[..., p, :, :], sigma(gammas, mu, nu))
    c *= 1j * kappa * csw
    return c.reshape(f.shape[:4] + (12, 12))


def clover_inverse(c):
    """C_inv = (1 + C)^-1 per site (App. A)."""
    return np.linalg.inv(np.eye(12) + c)


def spin5(x, gammas):
    return spin_mul(gamma5(gammas), x)


class CloverWilson:
    """D = 1 + C - kappa H on one gauge field, with A = C_inv D and the
    red/black domain blocks of Sec. 3.

    ``dims = (Lx, Ly, Lz, Lt)``; ``domain = (dx, dy, dz, dt)`` with every
    L_mu a multiple of 2 d_mu so that the colouring of domains by the parity of
    the sum of their indices is consistent across the periodic boundary.
    """

    def __init__(self, u, kappa, csw, gammas, bc_t=-1, domain=None):
        self.u = u
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.gammas = gammas
        self.bc_t = int(bc_t)
        self.dims = site_dims(u)
        self.c = clover_term(u, self.kappa, self.csw, gammas)
        self.cinv = clover_inverse(self.c)
        self.domain = None
        if domain is not None:
            self.set_domain(domain)

    # -- operator -----------------------------------------------------------
    def hop(self, x, fwd_mask=None, bwd_mask=None):
        return hop(self.u, x, self.gammas, self.bc_t, fwd_mask, bwd_mask)

    def D(self, x):
        """D x = x + C x - kappa H x."""
        return x + site_mul(self.c, x) - self.kappa * self.hop(x)

    def Ddag(self, x):
        """D^dag x = gamma_5 D gamma_5 x."""
        return spin5(self.D(spin5(x, self.gammas)), self.gammas)

    def A(self, x):
        """A x = C_inv D x = x - kappa C_inv H x (Eq. hoppingmat)."""
        return x - self.kappa * site_mul(self.cinv, self.hop(x))

    def apply_cinv(self, x):
        return site_mul(self.cinv, x)

    # -- domain decomposition (Sec. 3) --------------------------------------
    def set_domain(self, domain):
        domain = tuple(int(v) for v in domain)
        for mu in range(4):
            if self.dims[mu] % (2 * domain[mu]):
                raise ValueError("every L_mu must be a multiple of 2 d_mu")
        self.domain = domain
        lt, lz, ly, lx = self.u.shape[:4]
        t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                                 np.arange(lx), indexing="ij")
        coords = (x, y, z, t)
        self.colour = sum(coords[mu] // domain[mu] for mu in range(4)) % 2
        self.fwd_intra = [(coords[mu] % domain[mu] != domain[mu] - 1).astype(float)
                          for mu in range(4)]
        self.bwd_intra = [(coords[mu] % domain[mu] != 0).astype(float) for mu in range(4)]
        self.fwd_inter = [1.0 - m for m in self.fwd_intra]
        self.bwd_inter = [1.0 - m for m in self.bwd_intra]

    def mask(self, col):
        """0/1 site array of the sites in domains of colour ``col`` (0 = E, 1 = O)."""
        return (self.colour == col).astype(float)[..., None, None]

    def A_block(self, x, row, col):
        """The (row, col) block of A: A_EE, A_OO (row == col) or A_EO, A_OE.

        The result lives on the sites of colour ``row`` (zero elsewhere); only
        the components of x on colour ``col`` are read.
        """
        pr, pc = self.mask(row), self.mask(col)
        xc = pc * x
        if row == col:
            h = self.hop(xc, self.fwd_intra, self.bwd_intra)
            return pr * (xc - self.kappa * site_mul(self.cinv, h))
        h = self.hop(xc, self.fwd_inter, self.bwd_inter)
        return pr * (-self.kappa * site_mul(self.cinv, h))

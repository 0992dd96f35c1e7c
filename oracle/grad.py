"""Gradients of L = Re(eta^dag D^-1 b), float64.

With x = D^-1 b and lambda = D^-dag eta = gamma_5 D^-1 gamma_5 eta:

* dL = Re(lambda^dag db), so the gradient with respect to b is lambda;
* dL = -Re(lambda^dag dD x) with dD = dC - kappa dH.  Writing the result
  as dL = sum_links Re tr(G^dag dU):
    - hopping part (App. A, T+/- of every link):
      G_mu(y) += kappa sum_spin [(1 - g_mu) lambda(y)] (x) x(y + mu)^dag
      G_mu(y) += kappa sum_spin x(y) (x) [(1 + g_mu) lambda(y + mu)]^dag
      (the antiperiodic sign rides on the shifted spinors);
    - clover part: for each plane p and site n the colour matrix
      Z_p = sum_{alpha beta} sigma_p[alpha, beta] x_beta lambda_alpha^dag enters
      as dL = Re tr(dQ_p V_p) with V_p = (W - W^dag)/8, W = -i kappa c_SW Z_p;
      every link factor of every leaf of Q_p(n) then receives R or R^dag,
      R being the rest of the leaf product read cyclically through V_p.
* su(3) projection: Pi = TA(G U^dag), TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6,
  so that dL/dh = Re tr(Pi^dag X) for U -> exp(h X) U, X in su(3).
"""

import numpy as np

from .dirac import AXIS, dag, link_at, shift_fwd, spin_mul
from .gamma import PLANES, gamma5, sigma
from .solvers import bicgstab


def leaf_factors(mu, nu):
    """The four leaves of Q_{mu nu}(n) as (direction, offset, daggered) factors."""
    return (
        ((mu, {}, False), (nu, {mu: 1}, False), (mu, {nu: 1}, True), (nu, {}, True)),
        ((nu, {}, False), (mu, {mu: -1, nu: 1}, True), (nu, {mu: -1}, True), (mu, {mu: -1}, False)),
        ((mu, {mu: -1}, True), (nu, {mu: -1, nu: -1}, True), (mu, {mu: -1, nu: -1}, False),
         (nu, {nu: -1}, False)),
        ((nu, {nu: -1}, True), (mu, {nu: -1}, False), (nu, {mu: 1, nu: -1}, False), (mu, {}, True)),
    )


def _factor(u, d, off, is_dag):
    m = link_at(u[..., d, :, :], off)
    return dag(m) if is_dag else m


def _move_to(field, off):
    """Value computed at site n is stored at site n + off."""
    out = field
    for d, s in off.items():
        if s:
            out = np.roll(out, s, axis=AXIS[d])
    return out


def hop_force(op, x, lam):
    """Raw hopping-term gradient G_hop, ``[t][z][y][x][mu][3][3]``."""
    g = np.zeros(op.u.shape, dtype=np.complex128)
    eye = np.eye(4)
    for mu in range(4):
        xf = shift_fwd(x, mu, op.bc_t)
        lf = shift_fwd(lam, mu, op.bc_t)
        a = spin_mul(eye - op.gammas[mu], lam)
        g1 = np.einsum("...as,...bs->...ab", a, xf.conj())
        b = spin_mul(eye + op.gammas[mu], lf)
        g2 = np.einsum("...as,...bs->...ab", x, b.conj())
        g[..., mu, :, :] = op.kappa * (g1 + g2)
    return g


def clover_force(op, x, lam):
    """Raw clover-term gradient G_clov, ``[t][z][y][x][mu][3][3]``."""
    g = np.zeros(op.u.shape, dtype=np.complex128)
    for mu, nu in PLANES:
        s = sigma(op.gammas, mu, nu)
        z = np.einsum("...bj,ij,...ai->...ba", x, s, lam.conj())
        w = -1j * op.kappa * op.csw * z
        v = (w - dag(w)) / 8.0
        for leaf in leaf_factors(mu, nu):
            mats = [_factor(op.u, d, off, dg) for d, off, dg in leaf]
            for k, (d, off, dg) in enumerate(leaf):
                # R_k = A_{k+1} ... A_4 V A_1 ... A_{k-1}
                r = np.broadcast_to(np.eye(3), v.shape).astype(np.complex128)
                for m in mats[k + 1:]:
                    r = r @ m
                r = r @ v
                for m in mats[:k]:
                    r = r @ m
                contrib = r if dg else dag(r)
                g[..., d, :, :] += _move_to(contrib, off)
    return g


def solve_D(op, b, tol=1e-13, maxiter=5000):
    x, _, ok = bicgstab(op.D, b, tol, maxiter)
    if not ok:
        raise RuntimeError("oracle BiCGStab did not converge")
    return x


def solve_Ddag(op, eta, tol=1e-13, maxiter=5000):
    """lambda = D^-dag eta = gamma_5 D^-1 gamma_5 eta."""
    g5 = gamma5(op.gammas)
    return spin_mul(g5, solve_D(op, spin_mul(g5, eta), tol, maxiter))


def loss(op, eta, b, x=None):
    if x is None:
        x = solve_D(op, b)
    return float(np.vdot(eta.ravel(), x.ravel()).real)


def gradients(op, eta, b, tol=1e-13):
    """(grad_b, G_raw) of L = Re(eta^dag D^-1 b)."""
    x = solve_D(op, b, tol)
    lam = solve_Ddag(op, eta, tol)
    g = hop_force(op, x, lam) + clover_force(op, x, lam)
    return lam, g


def traceless_antihermitian(m):
    a = (m - dag(m)) / 2.0
    tr = np.trace(a, axis1=-2, axis2=-1)
    return a - tr[..., None, None] / 3.0 * np.eye(3)


def project_su3(g, u):
    """Pi = TA(G U^dag) per link."""
    return traceless_antihermitian(g @ dag(u))

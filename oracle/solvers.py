"""Krylov solvers: plain BiCGStab, Algorithm 5 and Algorithm 4 (Sec. 3).

Inner products are <a|b> = a^dag b (conjugate on the left).
"""

import numpy as np

from . import sap


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.vdot(a.ravel(), a.ravel()).real)


def bicgstab(apply, b, tol, maxiter, x0=None, record=None):
    """Textbook BiCGStab for apply(x) = b with r~ = r_0; float64.

    Returns (x, iterations, converged).  This is the reference solution of
    D x = b against which every preconditioned solve is compared.
    ``record`` (a list) receives (alpha, omega, x, r) per iteration when
    given.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x)
    rt = r.copy()
    bn = np.sqrt(norm2(b))
    if bn == 0:
        return x, 0, True
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_old = alpha = omega = 1.0
    for it in range(1, maxiter + 1):
        rho = vdot(rt, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho / vdot(rt, v)
        s = r - alpha * v
        t = apply(s)
        omega = vdot(t, s) / vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        if record is not None:
            record.append((alpha, omega, x.copy(), r.copy()))
        if np.sqrt(norm2(r)) / bn < tol:
            return x, it, True
    return x, maxiter, False


def bicgstab_precdd(op, b, n_sap, n_jac, tol, maxiter, record=None):
    """Algorithm 5: BiCGStab on (A M_SAP) y = b, then x = M_SAP y.

    Returns (x, y, iterations, status) with status "converged",
    "breakdown" or "maxiter".  ``record`` (a list) receives
    (alpha, omega, rnorm2) per iteration when given.
    """
    am = lambda v: sap.am_sap(op, v, n_sap, n_jac)
    x = np.zeros_like(b)
    r = b.copy()
    p = b.copy()
    rt = b.copy()
    bnorm2 = norm2(b)
    rho0 = bnorm2
    status = "maxiter"
    it = 0
    if bnorm2 == 0:
        return x, x.copy(), 0, "converged"
    for it in range(1, maxiter + 1):
        q = am(p)
        rtq = vdot(rt, q)
        if rtq == 0:
            status = "breakdown"
            break
        alpha = rho0 / rtq
        x = x + alpha * p
        r = r - alpha * q
        rnorm2 = norm2(r)
        if np.sqrt(rnorm2 / bnorm2) < tol:                      # first exit
            if record is not None:
                record.append((alpha, None, rnorm2))
            status = "converged"
            break
        t = am(r)
        tt = norm2(t)
        if tt == 0:
            status = "breakdown"
            break
        omega = vdot(t, r) / tt
        x = x + omega * r
        r = r - omega * t
        rnorm2 = norm2(r)
        rho = vdot(rt, r)
        if record is not None:
            record.append((alpha, omega, rnorm2))
        if np.sqrt(rnorm2 / bnorm2) < tol:                      # second exit
            status = "converged"
            break
        if rho == 0 or omega == 0:
            status = "breakdown"
            break
        beta = alpha * rho / (rho0 * omega)
        rho0 = rho
        p = r + beta * (p - omega * q)
    y = x
    return sap.msap(op, y, n_sap, n_jac), y, it, status


def to_single(v):
    """R_SP: round to complex64 (two float32)."""
    return v.astype(np.complex64)


def to_double(v):
    """P_DP: widen to complex128."""
    return v.astype(np.complex128)


def dci(op, b, tol, inner, max_outer=20, single=True):
    """Algorithm 4, defect correction for D x = b with an inner solver.

    ``inner(p)`` returns an approximate solution q of D q = p.  With
    ``single`` the inner right-hand side is rounded to single precision and
    the inner result is widened again, as R_SP / P_DP do.  The residual is
    recomputed as r = b - D x in float64 each step (the first of the two
    forms Algorithm 4 allows).  Returns (x, outer iterations, converged,
    relative residual history).
    """
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.sqrt(norm2(b))
    err = bn
    hist = []
    if bn == 0:
        return x, 0, True, hist
    for k in range(1, max_outer + 1):
        p = r / err
        if single:
            p = to_single(p)
        q = inner(p)
        dx = err * (to_double(q) if single else q)
        x = x + dx
        r = b - op.D(x)
        err = np.sqrt(norm2(r))
        hist.append(err / bn)
        if err / bn < tol:
            return x, k, True, hist
    return x, max_outer, False, hist


def sap_inner(op, n_sap, n_jac, tol, maxiter):
    """Inner solver for Algorithm 4: D q = p through A q = C_inv p with Algorithm 5."""
    def inner(p):
        p = to_double(p)
        x, _, _, _ = bicgstab_precdd(op, op.apply_cinv(p), n_sap, n_jac, tol, maxiter)
        return x
    return inner

"""Seeded generators for gauge fields, gauge transformations and sources.

Recipe (the synthetic stand-in for a thermalised ensemble; the paper names
no gauge configuration):

* every link is ``U = exp(i * eps * H)`` with ``H = sum_a h_a lambda_a / 2``,
  ``h_a ~ N(0, 1)`` and ``lambda_a`` the eight Gell-Mann matrices, so ``U`` is
  in SU(3) and ``eps`` sets the roughness (eps = 0 is the free field);
* draws come from ``numpy.random.Generator(PCG64(seed))`` in the order
  ``[t][z][y][x][mu][a]``;
* the exponential is taken through the eigendecomposition of the Hermitian
  ``H`` in float64;
* Gaussian sources draw the real and the imaginary part of every component
  from N(0, 1) with their own seed, in the order ``[t][z][y][x][colour][spin][re, im]``.
"""

import numpy as np


def lattice_shape(dims):
    """numpy shape ``(Lt, Lz, Ly, Lx)`` for ``dims = (Lx, Ly, Lz, Lt)``."""
    lx, ly, lz, lt = (int(v) for v in dims)
    return (lt, lz, ly, lx)


def gellmann_matrices():
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1] = -1j
    l[1, 1, 0] = 1j
    l[2, 0, 0] = 1
    l[2, 1, 1] = -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2] = -1j
    l[4, 2, 0] = 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2] = -1j
    l[6, 2, 1] = 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def _expi_hermitian(h, eps):
    """exp(i eps h) for a stack of Hermitian matrices via eigendecomposition."""
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, v.conj())


def _hermitian_from_coeffs(coef):
    return np.einsum("...a,aij->...ij", coef, gellmann_matrices() / 2)


def random_su3_field(dims, eps, seed):
    """Gauge field ``[t][z][y][x][mu][3][3]`` with links exp(i eps H)."""
    shape = lattice_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    coef = rng.standard_normal(shape + (4, 8))
    u = _expi_hermitian(_hermitian_from_coeffs(coef), float(eps))
    eye = np.eye(3)
    unit_err = np.abs(np.einsum("...ki,...kj->...ij", u.conj(), u) - eye).max()
    det_err = np.abs(np.linalg.det(u) - 1).max()
    if unit_err > 1e-13 or det_err > 1e-13:
        raise RuntimeError("generated links are not SU(3) to 1e-13")
    return u


def random_su3_field_fast(dims, eps, seed, device="cuda", chunk=1 << 15):
    """Same draws as ``random_su3_field``; the exponential exp(i eps H) is taken
    on ``device`` with torch's batched Hermitian eigendecomposition (float64),
    in chunks of ``chunk`` links, which makes 48^4 and 64^4 fields practical.
    Returns a numpy complex128 array in the canonical layout."""
    import torch

    shape = lattice_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    coef = rng.standard_normal(shape + (4, 8)).reshape(-1, 8)
    lam = torch.from_numpy(gellmann_matrices() / 2).to(device)
    out = np.empty((coef.shape[0], 3, 3), dtype=np.complex128)
    for a in range(0, coef.shape[0], chunk):
        c = torch.from_numpy(coef[a:a + chunk]).to(device=device, dtype=torch.complex128)
        h = (c @ lam.reshape(8, 9)).reshape(-1, 3, 3)
        w, v = torch.linalg.eigh(h)
        ph = torch.exp(1j * float(eps) * w.to(torch.complex128))
        u = (v * ph.unsqueeze(-2)) @ v.conj().transpose(-1, -2)
        out[a:a + chunk] = u.cpu().numpy()
    return out.reshape(shape + (4, 3, 3))


def random_su3_sites(dims, seed, eps=3.0):
    """One SU(3) matrix per site, ``[t][z][y][x][3][3]`` (a gauge transformation)."""
    shape = lattice_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    coef = rng.standard_normal(shape + (8,))
    return _expi_hermitian(_hermitian_from_coeffs(coef), float(eps))


def random_su3_algebra(shape, seed):
    """Random traceless anti-Hermitian 3x3 matrices (su(3) directions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    coef = rng.standard_normal(tuple(shape) + (8,))
    return 1j * _hermitian_from_coeffs(coef)


def gaussian_spinor(dims, seed, nrhs=None):
    """Gaussian quark field ``[t][z][y][x][3][4]`` (or ``[nrhs][...]``)."""
    shape = lattice_shape(dims) + (3, 4)
    if nrhs is not None:
        shape = (int(nrhs),) + shape
    rng = np.random.Generator(np.random.PCG64(seed))
    ri = rng.standard_normal(shape + (2,))
    return ri[..., 0] + 1j * ri[..., 1]


def point_source(dims, colour, spin, site=(0, 0, 0, 0)):
    """Unit source at ``site = (x, y, z, t)``, one colour and one spin."""
    out = np.zeros(lattice_shape(dims) + (3, 4), dtype=np.complex128)
    x, y, z, t = site
    out[t, z, y, x, colour, spin] = 1.0
    return out

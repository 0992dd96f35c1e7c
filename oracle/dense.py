"""Brute-force dense matrices, built one site and one hop at a time.

Independent of ``dirac.hop``: no array shifts, no einsum -- explicit Python
loops over sites and directions that place each 12x12 block of
D = 1 + C - kappa sum_mu (T+_mu + T-_mu) (App. A) at its (row, column)
position.  Only for tiny lattices (2^4: 192 x 192, 4^4: 3072 x 3072).

Vector index of (site n, colour a, spin alpha) = 12 n + 4 a + alpha with
n = ((t Lz + z) Ly + y) Lx + x, i.e. the canonical layout flattened.
"""

import itertools

import numpy as np


def site_index(coord, dims):
    x, y, z, t = coord
    lx, ly, lz, lt = dims
    return ((t * lz + z) * ly + y) * lx + x


def dense_D(u, c, kappa, gammas, bc_t):
    """Dense D from links ``u`` and per-site clover matrices ``c`` (12x12)."""
    lt, lz, ly, lx = u.shape[:4]
    dims = (lx, ly, lz, lt)
    v = lx * ly * lz * lt
    mat = np.zeros((12 * v, 12 * v), dtype=np.complex128)
    eye4 = np.eye(4)
    for t, z, y, x in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        n = (x, y, z, t)
        i = site_index(n, dims)
        rows = slice(12 * i, 12 * i + 12)
        mat[rows, rows] += np.eye(12) + c[t, z, y, x]
        for mu in range(4):
            # forward neighbour m = n + mu, block (1 - gamma_mu) U_mu(n)
            m = list(n)
            m[mu] += 1
            sign = 1.0
            if m[mu] == dims[mu]:
                m[mu] = 0
                if mu == 3:
                    sign = bc_t
            j = site_index(m, dims)
            blk = np.kron(u[t, z, y, x, mu], eye4 - gammas[mu])
            mat[rows, 12 * j:12 * j + 12] += -kappa * sign * blk
            # backward neighbour m = n - mu, block (1 + gamma_mu) U_mu(m)^dag
            m = list(n)
            m[mu] -= 1
            sign = 1.0
            if m[mu] < 0:
                m[mu] = dims[mu] - 1
                if mu == 3:
                    sign = bc_t
            j = site_index(m, dims)
            mx, my, mz, mt = m
            blk = np.kron(u[mt, mz, my, mx, mu].conj().T, eye4 + gammas[mu])
            mat[rows, 12 * j:12 * j + 12] += -kappa * sign * blk
    return mat


def flatten(psi):
    return psi.reshape(-1)


def unflatten(vec, like):
    return vec.reshape(like.shape)


def colour_of_sites(dims, domain):
    """Domain colour (0 = E, 1 = O) of every site, in flattened site order."""
    lx, ly, lz, lt = dims
    out = np.zeros(lx * ly * lz * lt, dtype=int)
    for t, z, y, x in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        n = (x, y, z, t)
        out[site_index(n, dims)] = sum(n[mu] // domain[mu] for mu in range(4)) % 2
    return out


def domain_of_sites(dims, domain):
    """A label per site that is equal exactly for sites in the same domain."""
    lx, ly, lz, lt = dims
    out = np.zeros(lx * ly * lz * lt, dtype=int)
    nd = [dims[mu] // domain[mu] for mu in range(4)]
    for t, z, y, x in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        n = (x, y, z, t)
        d = [n[mu] // domain[mu] for mu in range(4)]
        out[site_index(n, dims)] = ((d[3] * nd[2] + d[2]) * nd[1] + d[1]) * nd[0] + d[0]
    return out

"""Per-site flop model of the SAP-BiCGStab iteration (Sec. 4, Tables 2-3).

The paper reports, per MPI process, the flop count of 500 BiCGStab
iterations (Table 2) and of the A_EE + A_OO region inside them (Table 3)
without printing the model behind them.  The model below reproduces all ten
entries exactly when the loop count of Algorithm 1 is 4, Algorithm 2 applies
A_EE twice and each process block is split into two domains along x:

* a spatial hop costs 168 flop and a temporal hop 156 (in the paper's basis
  (1 -/+ gamma_4) is diagonal), so the full hopping term is 1320 flop;
* applying C_inv and forming x - kappa(...) costs 600 flop per site;
* f_in  = 600 + sum_mu 2 (1 - 1/d_mu) h_mu    (A_EE on a domain, per site)
* f_out = sum_mu (2 / d_mu) h_mu + 600 s      (A_EO, s = share of surface sites)
* per BiCGStab iteration and site:
  2 (n_sap + 1) [f_in + n_jac (f_in + 48) + f_out] + 96 n_sap + 48 + 1008,
  plus 42 flop per process for the scalar work.

The Dirac operator itself is counted with the conventional 1824 flop per site
(1320 for the hopping term + 504 for the clover term).
"""

from fractions import Fraction

HOP_SPACE = 168
HOP_TIME = 156
CLOVER_APPLY = 600
D_FLOP_PER_SITE = 1824


def f_in(domain, hops=(HOP_SPACE, HOP_SPACE, HOP_SPACE, HOP_TIME)):
    return CLOVER_APPLY + sum(2 * (1 - Fraction(1, d)) * h for d, h in zip(domain, hops))


def surface_share(domain):
    inner = 1
    vol = 1
    for d in domain:
        inner *= max(d - 2, 0)
        vol *= d
    return 1 - Fraction(inner, vol)


def f_out(domain, hops=(HOP_SPACE, HOP_SPACE, HOP_SPACE, HOP_TIME)):
    return sum(Fraction(2, d) * h for d, h in zip(domain, hops)) + CLOVER_APPLY * surface_share(domain)


def flop_per_site_iter(domain, n_sap, n_jac, hops=(HOP_SPACE, HOP_SPACE, HOP_SPACE, HOP_TIME)):
    fi = f_in(domain, hops)
    fo = f_out(domain, hops)
    return 2 * (n_sap + 1) * (fi + n_jac * (fi + 48) + fo) + 96 * n_sap + 48 + 1008


def table2_flop(block, n_sap=4, n_jac=2, iters=500):
    """Flop of ``iters`` iterations on one process block (Table 2 column)."""
    domain = (block[0] // 2,) + tuple(block[1:])
    vol = block[0] * block[1] * block[2] * block[3]
    per_iter = flop_per_site_iter(domain, n_sap, n_jac) * vol + 42
    return iters * per_iter


def table3_flop(block, n_sap=4, iters=500):
    """Flop of the A_EE + A_OO region (Table 3 column)."""
    domain = (block[0] // 2,) + tuple(block[1:])
    vol = block[0] * block[1] * block[2] * block[3]
    return iters * 2 * (n_sap + 1) * f_in(domain) * vol

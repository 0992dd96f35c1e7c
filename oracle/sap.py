"""SAP preconditioner with Jacobi domain inverses (Sec. 3, Algorithms 1-3).

All vectors are full-lattice quark fields; a vector "on E" is zero on the
odd-coloured domains.  Colour 0 is E, colour 1 is O.

Readings (Sec. 3 leaves these open):

* ``n_sap`` is the loop count of Algorithm 1, whose closing lines add one
  more sweep, so K is applied n_sap + 1 times:
  M_SAP = K sum_{j=0}^{n_sap} (1 - A K)^j;
* ``n_jac`` is the number of A_EE applications in Algorithm 2, which gives
  B_EE = sum_{j=0}^{n_jac} (I - A_EE)^j (n_jac >= 1);
* Algorithm 3 is taken to return A (M_SAP b); its garbled lines that write
  "A_EE s_E" / "A_OO s_O" are the domain inverses B_EE, B_OO of the final
  sweep (the flop count of Tables 2-3 requires n_sap + 1 calls of the
  Jacobi routine per colour).
"""

import numpy as np

E, O = 0, 1


def jacobi(op, b, col, n_jac):
    """x = B b on the domains of colour ``col`` (Algorithm 2).

    q = A_cc b;  x = 2 b - q;  then n_jac - 1 times: q = A_cc x;  x = x + b - q.
    """
    if n_jac < 1:
        raise ValueError("n_jac >= 1")
    b = op.mask(col) * b
    q = op.A_block(b, col, col)
    x = 2 * b - q
    for _ in range(1, n_jac):
        q = op.A_block(x, col, col)
        x = x + b - q
    return x


def msap(op, b, n_sap, n_jac):
    """x = M_SAP b (Algorithm 1): n_sap red/black sweeps plus a closing sweep."""
    me, mo = op.mask(E), op.mask(O)
    s = b.copy()
    for _ in range(n_sap):
        x_e = jacobi(op, s, E, n_jac)
        q_e = op.A_block(x_e, E, E)
        s = s + me * (b - q_e)                  # s_E = s_E + b_E - q_E
        s = s - op.A_block(x_e, O, E)           # s_O = s_O - A_OE x_E
        x_o = jacobi(op, s, O, n_jac)
        q_o = op.A_block(x_o, O, O)
        s = s + mo * (b - q_o)                  # s_O = s_O + b_O - q_O
        s = s - op.A_block(x_o, E, O)           # s_E = s_E - A_EO x_O
    x_e = jacobi(op, s, E, n_jac)
    s = s - op.A_block(x_e, O, E)
    x_o = jacobi(op, s, O, n_jac)
    return x_e + x_o


def am_sap(op, b, n_sap, n_jac):
    """x = A M_SAP b (Algorithm 3, read as A applied to the result of Algorithm 1)."""
    return op.A(msap(op, b, n_sap, n_jac))


def k_apply(op, b, n_jac, exact=None):
    """K b with K = [[B_EE, 0], [-B_OO A_OE B_EE, B_OO]] (Eq. Msap).

    ``exact`` may supply a function (vector, colour) -> exact A_cc^-1 vector.
    """
    inv = exact if exact is not None else (lambda v, c: jacobi(op, v, c, n_jac))
    y_e = inv(op.mask(E) * b, E)
    y_o = inv(op.mask(O) * b - op.A_block(y_e, O, E), O)
    return y_e + y_o


def msap_series(op, b, n_sap, n_jac):
    """K sum_{j=0}^{n_sap} (1 - A K)^j b, the closed form of Eq. Msap."""
    v = b.copy()
    acc = np.zeros_like(b)
    for _ in range(n_sap + 1):
        acc = acc + v
        v = v - op.A(k_apply(op, v, n_jac))
    return k_apply(op, acc, n_jac)

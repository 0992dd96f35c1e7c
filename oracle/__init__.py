"""Plain float64 CPU oracle for the Clover-Wilson SAP-BiCGStab quark solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library; the two meet only in the seeded generators of
``lattice_inputs``.

Everything here is written for a reader to check against the paper by eye:
numpy array expressions over whole lattices, complex128 throughout, no
blocking, no fusion, no reordering of the algorithms' steps.

Modules and the passages they follow (arXiv:2109.10687):

* ``gamma``   -- gamma matrices of App. A, sigma_{mu nu}, gamma_5 and the
  rotation to the chiral basis;
* ``dirac``   -- hopping term, four-leaf field strength, clover term, its
  inverse, D = 1 + C - kappa H (App. A), A = C_inv D (Eq. hoppingmat of
  Sec. 3), and the red/black domain blocks A_EE, A_OO, A_EO, A_OE (Sec. 3);
* ``sap``     -- Jacobi domain inverse (Algorithm 2), the SAP preconditioner
  (Algorithm 1), A M_SAP (Algorithm 3) and the dense K of Eq. Msap;
* ``solvers`` -- plain BiCGStab on D (the reference solution), the
  preconditioned BiCGStab of Algorithm 5 and the defect-correction loop of
  Algorithm 4;
* ``grad``    -- gradients of L = Re(eta^dag D^-1 b) with respect to b and U;
* ``dense``   -- brute-force dense matrices built site by site with Python
  loops (tiny lattices only), an independent check of the stencil;
* ``flops``   -- the per-site flop model that reproduces Tables 2 and 3.

Parity pins: every function above is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; iteration counts and times are "parity unpinned"
because the paper prints none.
"""

"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws random numbers and assembles them into fields in the
canonical external layout.  It holds none of the solver's arithmetic (no
Dirac operator, no clover term, no preconditioner): both sides of every
parity test take their inputs from here and compute everything else on their
own.

Canonical layout (the one the paper quotes for the K computer, Sec. 4):

* lattice extents are given as ``dims = (Lx, Ly, Lz, Lt)``; numpy arrays are
  indexed ``[t][z][y][x]`` so that x runs fastest;
* a quark field is complex ``[t][z][y][x][colour 3][spin 4]``;
* a gauge field is complex ``[t][z][y][x][mu 4][row 3][col 3]`` with
  ``mu = 0, 1, 2, 3`` for the x, y, z, t directions.
"""

from .fields import (  # noqa: F401
    gellmann_matrices,
    random_su3_field,
    random_su3_field_fast,
    random_su3_sites,
    gaussian_spinor,
    point_source,
    random_su3_algebra,
    lattice_shape,
)

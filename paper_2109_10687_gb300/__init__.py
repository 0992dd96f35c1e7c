"""GB300 (sm_103a) Clover-Wilson SAP-BiCGStab quark solver of arXiv:2109.10687.

The compute path is the C-ABI library libqcd_gb300.so (include/qcd_gb300.h),
built from ``csrc/*.cu`` by ``build.build()``.  ``binding`` exposes its
entry points under the same names; ``lattice.Lattice`` wraps a context for
torch users; ``autograd`` provides the differentiable solve.
"""

__all__ = ["binding", "build", "lattice", "autograd"]

"""The allocation-free |a|^2 entry point (qcd_norm2_noalloc), called through
the C ABI, against the workspace-based qcd_norm2 on the same fields.

qcd_norm2_noalloc serves callers that must not allocate device memory during
the call (a caching allocator or memory pool owning the free memory, code
that must avoid the synchronisation an allocation can cause); it keeps its
scratch in a static device array inside the library.  This file is collected
last so that a failure here stops a -x run only after every other test ran.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_norm2_noalloc_matches_norm2_twice():
    from gpu_util import Problem
    from lattice_inputs import gaussian_spinor
    from paper_2109_10687_gb300 import binding as B

    p = Problem((8, 8, 8, 8), (4, 4, 4, 4), seed=4001, oracle=False)
    try:
        nrhs = 3
        x = gaussian_spinor(p.dims, 4002, nrhs=nrhs)
        for prec in (B.PREC_SINGLE, B.PREC_DOUBLE):
            name = "single" if prec == B.PREC_SINGLE else "double"
            buf = p.lat.to_internal(x, name, nrhs)
            ref = np.array([np.vdot(x[r].ravel(), x[r].ravel()).real for r in range(nrhs)])
            for _ in range(2):  # two calls in a row share the static scratch
                got = np.array(B.qcd_norm2_noalloc(p.lat.ctx, buf, prec, nrhs))
                want = np.array(B.qcd_norm2(p.lat.ctx, buf, prec, nrhs))
                assert np.allclose(got, want, rtol=1e-12, atol=0)
                assert np.allclose(got, ref, rtol=1e-6, atol=0)
        # beyond the static scratch: a clear argument error, nothing launched
        big = p.lat.field("single", 17)
        with pytest.raises(B.QcdError) as e:
            B.qcd_norm2_noalloc(p.lat.ctx, big, B.PREC_SINGLE, 17)
        assert e.value.code == B.QCD_ERR_ARG
    finally:
        p.close()

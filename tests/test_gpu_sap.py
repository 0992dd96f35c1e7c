"""GPU parity of the SAP preconditioner (Algorithms 1-3) against the oracle's
literal Algorithms, float32 and float16 storage."""

import numpy as np
import pytest

from gpu_util import Problem, rel_l2, to_np
from oracle import sap

pytestmark = pytest.mark.gpu

CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4)),
    ((4, 4, 4, 8), (2, 2, 2, 2)),
    ((8, 8, 4, 8), (2, 4, 2, 4)),
    ((2, 2, 2, 2), (1, 1, 1, 1)),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])) + "_d" + "".join(map(str, c[1])))
def prob(request):
    dims, domain = request.param
    p = Problem(dims, domain, eps=0.3, kappa=0.12, csw=1.0, seed=1101)
    yield p
    p.close()


@pytest.mark.parametrize("n_sap,n_jac", [(0, 1), (1, 2), (4, 4)])
def test_msap_float32(prob, n_sap, n_jac):
    b = prob.source(2101)
    got = to_np(prob.lat.sap(b, n_sap, n_jac, "single"))
    ref = sap.msap(prob.op, b, n_sap, n_jac)
    assert rel_l2(got, ref) <= 1e-5


def test_am_sap_float32(prob):
    b = prob.source(2102)
    got = to_np(prob.lat.sap(b, 4, 4, "single", with_A=True))
    ref = sap.am_sap(prob.op, b, 4, 4)
    assert rel_l2(got, ref) <= 1e-5


def test_msap_float16_storage(prob):
    """float16 storage with per-site norms: an approximation of M_SAP at the
    level of half-precision rounding (2^-11 per stored value)."""
    b = prob.source(2103)
    got = to_np(prob.lat.sap(b, 4, 4, "half"))
    ref = sap.msap(prob.op, b, 4, 4)
    assert rel_l2(got, ref) <= 5e-3


def test_msap_float16_gauge_storage(prob):
    """float16 links and C_inv with float32 vectors: an approximation of M_SAP
    at the level of half-precision rounding of the operator."""
    b = prob.source(2105)
    got = to_np(prob.lat.sap(b, 4, 4, "half_gauge"))
    ref = sap.msap(prob.op, b, 4, 4)
    assert rel_l2(got, ref) <= 5e-3


def test_sap_reduces_residual(prob):
    """A M_SAP is close to the identity: |b - A M b| / |b| well below 1."""
    b = prob.source(2104)
    amb = to_np(prob.lat.sap(b, 4, 4, "single", with_A=True))
    assert rel_l2(amb, b) < 0.5

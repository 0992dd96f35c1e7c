"""A small object layer over the C ABI for torch users.

``Lattice`` owns one library context (one lattice, one gauge field, one
clover term) and moves canonical complex128 fields (numpy or torch, layout
``[rhs][t][z][y][x][colour][spin]``) in and out of the library's internal
device layout.  Every operation is a call into libqcd_gb300.
"""

import numpy as np
import torch

from . import binding as B

PREC = {"double": B.PREC_DOUBLE, "single": B.PREC_SINGLE, "half": B.PREC_HALF, "half_gauge": B.PREC_HALF_GAUGE,
        B.PREC_DOUBLE: B.PREC_DOUBLE, B.PREC_SINGLE: B.PREC_SINGLE, B.PREC_HALF: B.PREC_HALF,
        B.PREC_HALF_GAUGE: B.PREC_HALF_GAUGE}


def _canonical_real(t, device):
    """complex128 canonical field (numpy/torch) -> contiguous float64 torch view on ``device``."""
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(t))
    if t.is_complex():
        t = torch.view_as_real(t.to(torch.complex128).contiguous())
    return t.to(device=device, dtype=torch.float64).contiguous()


class Lattice:
    def __init__(self, dims, domain=(4, 4, 4, 4), bc_t=-1, basis="chiral", device="cuda"):
        self.dims = tuple(int(v) for v in dims)
        self.domain = tuple(int(v) for v in domain)
        self.device = torch.device(device)
        if self.device.type == "cuda":
            if self.device.index is None:
                self.device = torch.device("cuda", torch.cuda.current_device())
            torch.cuda.set_device(self.device)
        basis_code = B.BASIS_CHIRAL if basis == "chiral" else B.BASIS_PAPER
        self.ctx = B.qcd_create(self.dims, self.domain, bc_t, basis_code)
        lx, ly, lz, lt = self.dims
        self.site_shape = (lt, lz, ly, lx)
        self.kappa = None
        self.csw = None

    # -- set-up -------------------------------------------------------------
    def set_gauge(self, u, check_tol=1e-12):
        self._u = _canonical_real(u, self.device)
        B.qcd_set_gauge(self.ctx, self._u, check_tol)

    def set_params(self, kappa, csw):
        self.kappa, self.csw = float(kappa), float(csw)
        B.qcd_set_params(self.ctx, kappa, csw)

    def build_clover(self):
        B.qcd_build_clover(self.ctx)

    def setup(self, u, kappa, csw):
        self.set_gauge(u)
        self.set_params(kappa, csw)
        self.build_clover()
        return self

    # -- fields -------------------------------------------------------------
    def field(self, prec="single", nrhs=1):
        nbytes = B.qcd_field_bytes(self.ctx, PREC[prec], nrhs)
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def to_internal(self, psi, prec="single", nrhs=1):
        src = _canonical_real(psi, self.device)
        out = self.field(prec, nrhs)
        B.qcd_import_spinor(self.ctx, out, src, PREC[prec], nrhs)
        return out

    def to_canonical(self, buf, prec="single", nrhs=1):
        shape = ((nrhs,) if nrhs > 1 else ()) + self.site_shape + (3, 4, 2)
        out = torch.empty(shape, dtype=torch.float64, device=self.device)
        B.qcd_export_spinor(self.ctx, out, buf, PREC[prec], nrhs)
        return torch.view_as_complex(out)

    # -- operators on canonical fields ----------------------------------------
    def apply_D(self, psi, prec="single", dagger=False, nrhs=1):
        a = self.to_internal(psi, prec, nrhs)
        o = self.field(prec, nrhs)
        B.qcd_apply_D(self.ctx, o, a, PREC[prec], int(dagger), nrhs)
        return self.to_canonical(o, prec, nrhs)

    def apply_A(self, psi, nrhs=1):
        a = self.to_internal(psi, "single", nrhs)
        o = self.field("single", nrhs)
        B.qcd_apply_A(self.ctx, o, a, nrhs)
        return self.to_canonical(o, "single", nrhs)

    def apply_clover(self, psi, prec="single", inverse=False, nrhs=1):
        a = self.to_internal(psi, prec, nrhs)
        B.qcd_apply_clover(self.ctx, a, a, PREC[prec], int(inverse), nrhs)
        return self.to_canonical(a, prec, nrhs)

    def apply_A_block(self, psi, row, col):
        a = self.to_internal(psi, "single")
        o = self.field("single")
        B.qcd_apply_A_block(self.ctx, o, a, row, col)
        return self.to_canonical(o, "single")

    def sap(self, psi, n_sap, n_jac, sap_prec="single", with_A=False, nrhs=1):
        a = self.to_internal(psi, "single", nrhs)
        o = self.field("single", nrhs)
        if nrhs == 1:
            B.qcd_sap_apply(self.ctx, o, a, n_sap, n_jac, PREC[sap_prec], int(with_A))
        else:
            B.qcd_sap_apply_nrhs(self.ctx, o, a, nrhs, n_sap, n_jac, PREC[sap_prec], int(with_A))
        return self.to_canonical(o, "single", nrhs)

    def solve(self, b, nrhs=1, params=None, raise_on_error=True, host=False, **kw):
        """x with D x = b (canonical complex128 in, canonical complex128 out)."""
        p = params if params is not None else B.qcd_solve_params_default()
        for k, v in kw.items():
            setattr(p, k, PREC[v] if k == "sap_prec" else v)
        if host:
            src = np.ascontiguousarray(np.asarray(b, dtype=np.complex128)).view(np.float64)
            out = np.zeros_like(src)
        else:
            src = _canonical_real(b, self.device)
            out = torch.zeros_like(src)
        rc, info = B.qcd_solve(self.ctx, out, src, nrhs, p, raise_on_error=raise_on_error)
        if host:
            return out.view(np.complex128), rc, info
        return torch.view_as_complex(out), rc, info

    def close(self):
        if self.ctx is not None:
            B.qcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

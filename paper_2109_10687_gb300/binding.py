"""ctypes binding of libqcd_gb300 (include/qcd_gb300.h).

Argument marshalling only: every function below forwards to the C entry
point of the same name; all arithmetic runs in the library's CUDA kernels.
Tensors are torch tensors (device or pinned/host) or numpy arrays (host);
streams default to torch's current CUDA stream.  If the shared library has
not been built, loading it raises immediately -- there is no fallback.
"""

import ctypes
import os

import numpy as np

from . import build as _build

QCD_OK = 0
QCD_ERR_ARG = 1
QCD_ERR_CUDA = 2
QCD_ERR_OOM = 3
QCD_ERR_NOT_CONVERGED = 4
QCD_ERR_BREAKDOWN = 5
QCD_ERR_NONFINITE = 6
QCD_ERR_TIMEOUT = 7
QCD_ERR_STATE = 8

PREC_DOUBLE, PREC_SINGLE, PREC_HALF, PREC_HALF_GAUGE = 0, 1, 2, 3
BASIS_CHIRAL, BASIS_PAPER = 0, 1
KC_DSLASH, KC_SAP_BLOCK, KC_BLAS, KC_DOUBLE, KC_OTHER = range(5)

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_CONVERGED",
                5: "ERR_BREAKDOWN", 6: "ERR_NONFINITE", 7: "ERR_TIMEOUT", 8: "ERR_STATE"}


class QcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("n_sap", ctypes.c_int), ("n_jac", ctypes.c_int),
                ("sap_prec", ctypes.c_int), ("use_graph", ctypes.c_int), ("x_is_guess", ctypes.c_int),
                ("residual_prec", ctypes.c_int), ("outer_restart", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("status", ctypes.c_int),
                ("true_resid", ctypes.c_double), ("seconds", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes)
_SIGS = {
    "qcd_version": (ctypes.c_char_p, []),
    "qcd_create": (_I, [ctypes.POINTER(_I), ctypes.POINTER(_I), _I, _I, ctypes.POINTER(_P)]),
    "qcd_destroy": (_I, [_P]),
    "qcd_last_error": (ctypes.c_char_p, [_P]),
    "qcd_set_gauge": (_I, [_P, _P, _I, _D, _P]),
    "qcd_set_params": (_I, [_P, _D, _D]),
    "qcd_build_clover": (_I, [_P, _P]),
    "qcd_field_bytes": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "qcd_import_spinor": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "qcd_export_spinor": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "qcd_apply_D": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "qcd_apply_A": (_I, [_P, _P, _P, _I, _P]),
    "qcd_apply_clover": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "qcd_apply_A_block": (_I, [_P, _P, _P, _I, _I, _P]),
    "qcd_sap_apply": (_I, [_P, _P, _P, _I, _I, _I, _I, _P]),
    "qcd_sap_apply_nrhs": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P]),
    "qcd_norm2": (_I, [_P, ctypes.POINTER(_D), _P, _I, _I, _P]),
    "qcd_norm2_noalloc": (_I, [_P, ctypes.POINTER(_D), _P, _I, _I, _P]),
    "qcd_cdot": (_I, [_P, ctypes.POINTER(_D), _P, _P, _I, _I, _P]),
    "qcd_solve": (_I, [_P, _P, _P, _I, _I, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), _P]),
    "qcd_solve_params_default": (_I, [ctypes.POINTER(SolveParams)]),
    "qcd_grad": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, ctypes.POINTER(SolveParams), _P]),
    "qcd_profile_enable": (_I, [_P, _I]),
    "qcd_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D), _I]),
    "qcd_launch_count": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "qcd_set_tuning": (_I, [_P, _I]),
    "qcd_set_sap_shape": (_I, [_P, _I]),
    "qcd_set_link_compression": (_I, [_P, _I]),
    "qcd_link_format": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "qcd_set_sap_domain": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "qcd_tune_domain": (_I, [ctypes.POINTER(ctypes.c_int), _I, _I, _P, _P, _I, ctypes.c_double, ctypes.c_double,
                             ctypes.POINTER(SolveParams), ctypes.POINTER(ctypes.c_int), _I,
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "qcd_tune_domain_default_count": (_I, []),
    "qcd_batch_create": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "qcd_batch_destroy": (_I, [_P]),
    "qcd_batch_last_error": (ctypes.c_char_p, [_P]),
    "qcd_batch_apply_D": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P]),
    "qcd_batch_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, ctypes.POINTER(SolveParams),
                             ctypes.POINTER(SolveInfo), _P]),
    "qcd_batch_set_shared": (_I, [_P, _I]),
    "qcd_tuning_report": (_I, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "qcd_measure_fp32_peak": (_I, [_P, ctypes.POINTER(ctypes.c_double), _P]),
    "qcd_device_status": (_I, [_P, ctypes.POINTER(_I), _I, _P]),
    "qcd_test_inject": (_I, [_P, _I]),
}


def library_path():
    return _build.lib_path()


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
        dll = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(dll, name)
            fn.restype = res
            fn.argtypes = args
        _lib = dll
    return _lib


def exported_symbols():
    return list(_SIGS)


# -- marshalling helpers ---------------------------------------------------------

def _ptr(t):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _on_device(t):
    return 0 if isinstance(t, np.ndarray) else int(t.is_cuda)


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def check(ctx, rc):
    if rc != QCD_OK:
        raise QcdError(rc, lib().qcd_last_error(ctx).decode())
    return rc


# -- C entry points with the same names ---------------------------------------------

def qcd_version():
    return lib().qcd_version().decode()


def qcd_create(dims, domain=(4, 4, 4, 4), bc_t=-1, basis=BASIS_CHIRAL):
    d = (ctypes.c_int * 4)(*dims)
    dd = (ctypes.c_int * 4)(*domain)
    ctx = ctypes.c_void_p()
    rc = lib().qcd_create(d, dd, int(bc_t), int(basis), ctypes.byref(ctx))
    if rc != QCD_OK:
        raise QcdError(rc, lib().qcd_last_error(None).decode())
    return ctx


def qcd_destroy(ctx):
    return lib().qcd_destroy(ctx)


def qcd_set_gauge(ctx, u, check_tol=1e-12, stream=None):
    return check(ctx, lib().qcd_set_gauge(ctx, _ptr(u), _on_device(u), float(check_tol), _stream(stream)))


def qcd_set_params(ctx, kappa, csw):
    return check(ctx, lib().qcd_set_params(ctx, float(kappa), float(csw)))


def qcd_build_clover(ctx, stream=None):
    return check(ctx, lib().qcd_build_clover(ctx, _stream(stream)))


def qcd_field_bytes(ctx, prec, nrhs=1):
    n = ctypes.c_size_t()
    check(ctx, lib().qcd_field_bytes(ctx, int(prec), int(nrhs), ctypes.byref(n)))
    return n.value


def qcd_import_spinor(ctx, dst, src, prec, nrhs=1, stream=None):
    return check(ctx, lib().qcd_import_spinor(ctx, _ptr(dst), _ptr(src), int(prec), int(nrhs), _on_device(src),
                                              _stream(stream)))


def qcd_export_spinor(ctx, dst, src, prec, nrhs=1, stream=None):
    return check(ctx, lib().qcd_export_spinor(ctx, _ptr(dst), _ptr(src), int(prec), int(nrhs), _on_device(dst),
                                              _stream(stream)))


def qcd_apply_D(ctx, out, inp, prec, dagger=0, nrhs=1, stream=None):
    return check(ctx, lib().qcd_apply_D(ctx, _ptr(out), _ptr(inp), int(prec), int(dagger), int(nrhs),
                                        _stream(stream)))


def qcd_apply_A(ctx, out, inp, nrhs=1, stream=None):
    return check(ctx, lib().qcd_apply_A(ctx, _ptr(out), _ptr(inp), int(nrhs), _stream(stream)))


def qcd_apply_clover(ctx, out, inp, prec, inverse=0, nrhs=1, stream=None):
    return check(ctx, lib().qcd_apply_clover(ctx, _ptr(out), _ptr(inp), int(prec), int(inverse), int(nrhs),
                                             _stream(stream)))


def qcd_apply_A_block(ctx, out, inp, row, col, stream=None):
    return check(ctx, lib().qcd_apply_A_block(ctx, _ptr(out), _ptr(inp), int(row), int(col), _stream(stream)))


def qcd_sap_apply(ctx, out, inp, n_sap, n_jac, sap_prec=PREC_SINGLE, with_A=0, stream=None):
    return check(ctx, lib().qcd_sap_apply(ctx, _ptr(out), _ptr(inp), int(n_sap), int(n_jac), int(sap_prec),
                                          int(with_A), _stream(stream)))


def qcd_sap_apply_nrhs(ctx, out, inp, nrhs, n_sap, n_jac, sap_prec=PREC_SINGLE, with_A=0, stream=None):
    return check(ctx, lib().qcd_sap_apply_nrhs(ctx, _ptr(out), _ptr(inp), int(nrhs), int(n_sap), int(n_jac),
                                               int(sap_prec), int(with_A), _stream(stream)))


def qcd_norm2(ctx, a, prec=PREC_SINGLE, nrhs=1, stream=None):
    out = (ctypes.c_double * nrhs)()
    check(ctx, lib().qcd_norm2(ctx, out, _ptr(a), int(prec), int(nrhs), _stream(stream)))
    return list(out)


def qcd_norm2_noalloc(ctx, a, prec=PREC_SINGLE, nrhs=1, stream=None):
    """|a|^2 through the entry point that allocates no device memory."""
    out = (ctypes.c_double * nrhs)()
    check(ctx, lib().qcd_norm2_noalloc(ctx, out, _ptr(a), int(prec), int(nrhs), _stream(stream)))
    return list(out)


def qcd_cdot(ctx, a, b, prec=PREC_SINGLE, nrhs=1, stream=None):
    out = (ctypes.c_double * (2 * nrhs))()
    check(ctx, lib().qcd_cdot(ctx, out, _ptr(a), _ptr(b), int(prec), int(nrhs), _stream(stream)))
    return [complex(out[2 * i], out[2 * i + 1]) for i in range(nrhs)]


def qcd_solve_params_default():
    p = SolveParams()
    lib().qcd_solve_params_default(ctypes.byref(p))
    return p


def qcd_solve(ctx, x, b, nrhs=1, params=None, stream=None, raise_on_error=True):
    """Solve D x = b; returns (status, SolveInfo)."""
    p = params if params is not None else qcd_solve_params_default()
    info = SolveInfo()
    on_dev = _on_device(b)
    rc = lib().qcd_solve(ctx, _ptr(x), _ptr(b), int(nrhs), on_dev, ctypes.byref(p), ctypes.byref(info),
                         _stream(stream))
    if raise_on_error and rc != QCD_OK:
        raise QcdError(rc, lib().qcd_last_error(ctx).decode())
    return rc, info


def qcd_grad(ctx, eta, b, grad_b, grad_u, x=None, lam=None, project=0, params=None, stream=None):
    p = params if params is not None else qcd_solve_params_default()
    return check(ctx, lib().qcd_grad(ctx, _ptr(eta), _ptr(b), _ptr(x), _ptr(lam), _ptr(grad_b), _ptr(grad_u),
                                     int(project), ctypes.byref(p), _stream(stream)))


def qcd_profile_enable(ctx, enable=True):
    return check(ctx, lib().qcd_profile_enable(ctx, int(bool(enable))))


def qcd_profile_read(ctx, kernel_class, reset=False):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    check(ctx, lib().qcd_profile_read(ctx, int(kernel_class), ctypes.byref(n), ctypes.byref(ms), int(bool(reset))))
    return n.value, ms.value


def qcd_launch_count(ctx):
    n = ctypes.c_longlong()
    check(ctx, lib().qcd_launch_count(ctx, ctypes.byref(n)))
    return n.value


def qcd_set_link_compression(ctx, mode):
    """-1 autotuned (default), 0 never, 1 always: float32 D with 12-real links."""
    return check(ctx, lib().qcd_set_link_compression(ctx, int(mode)))


def qcd_link_format(ctx):
    """12 or 18: the link format the float32 operators use now."""
    r = ctypes.c_int()
    check(ctx, lib().qcd_link_format(ctx, ctypes.byref(r)))
    return r.value


def qcd_set_tuning(ctx, enable=True):
    return check(ctx, lib().qcd_set_tuning(ctx, int(bool(enable))))


def qcd_tune_domain(dims, u, b, kappa, csw, params=None, candidates=None, bc_t=-1, basis=0):
    """Time-to-solution autotuner over SAP domain shapes.  u, b: canonical
    float64 (real-view) tensors or arrays, both on the device or both on the
    host.  Returns (best_domain, {candidate: seconds or None})."""
    p = params if params is not None else qcd_solve_params_default()
    cands = [tuple(int(v) for v in c) for c in candidates] if candidates else None
    n = len(cands) if cands else 0
    flat = (ctypes.c_int * (4 * max(n, 1)))(*[v for c in (cands or []) for v in c])
    nout = n if n else lib().qcd_tune_domain_default_count()
    secs = (ctypes.c_double * nout)()
    best = (ctypes.c_int * 4)()
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    rc = lib().qcd_tune_domain(d, int(bc_t), int(basis), _ptr(u), _ptr(b), _on_device(b), float(kappa), float(csw),
                               ctypes.byref(p), flat if n else None, n, best, secs)
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_tune_domain: no candidate solved")
    keys = cands if cands else [None] * nout
    return tuple(best), {k if k else i: (v if v >= 0 else None) for i, (k, v) in enumerate(zip(keys, secs))}


def qcd_set_sap_domain(ctx, sdom):
    """SAP domains of any extents, independent of the storage blocking (None: the storage domains)."""
    arr = (ctypes.c_int * 4)(*[int(v) for v in sdom]) if sdom is not None else None
    return check(ctx, lib().qcd_set_sap_domain(ctx, arr))


def qcd_set_sap_shape(ctx, shape):
    """SAP block-kernel shape for 4^4 domains: -1 autotuned, 0 one site per
    thread, 1 two sites per thread."""
    return check(ctx, lib().qcd_set_sap_shape(ctx, int(shape)))


def qcd_measure_fp32_peak(ctx, stream=None):
    """float32 FMA throughput of the device in TFLOP/s (measured)."""
    v = ctypes.c_double()
    check(ctx, lib().qcd_measure_fp32_peak(ctx, ctypes.byref(v), _stream(stream)))
    return v.value


INJECT_NONE = 0
INJECT_STAGING_WAIT = 1
INJECT_HALO_WAIT = 2


def qcd_device_status(ctx, reset=False, stream=None):
    """The device status word (QCD_OK, or e.g. QCD_ERR_TIMEOUT)."""
    v = _I()
    check(ctx, lib().qcd_device_status(ctx, ctypes.byref(v), int(bool(reset)), _stream(stream)))
    return v.value


def qcd_test_inject(ctx, what):
    return check(ctx, lib().qcd_test_inject(ctx, int(what)))


def qcd_tuning_report(ctx):
    buf = ctypes.create_string_buffer(4096)
    check(ctx, lib().qcd_tuning_report(ctx, buf, len(buf)))
    return buf.value.decode()


def _batch_check(batch, rc):
    if rc != QCD_OK:
        raise QcdError(rc, lib().qcd_batch_last_error(batch).decode())
    return rc


def qcd_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    out = ctypes.c_void_p()
    rc = lib().qcd_batch_create(len(ctxs), arr, ctypes.byref(out))
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_batch_create failed")
    return out


def qcd_batch_destroy(batch):
    return lib().qcd_batch_destroy(batch)


def qcd_batch_apply_D(batch, outs, ins, dagger=0, stream=None):
    o = (ctypes.c_void_p * len(outs))(*[_ptr(t) for t in outs])
    i = (ctypes.c_void_p * len(ins))(*[_ptr(t) for t in ins])
    return _batch_check(batch, lib().qcd_batch_apply_D(batch, o, i, int(dagger), _stream(stream)))


def qcd_batch_set_shared(batch, enable=True):
    """1: qcd_batch_solve in shared launches where supported; 0: concurrent per-lattice solves."""
    return _batch_check(batch, lib().qcd_batch_set_shared(batch, int(bool(enable))))


def qcd_batch_solve(batch, xs, bs, params=None, stream=None, raise_on_error=True):
    """Solve every lattice of the batch; returns (status, [SolveInfo])."""
    p = params if params is not None else qcd_solve_params_default()
    n = len(xs)
    xa = (ctypes.c_void_p * n)(*[_ptr(t) for t in xs])
    ba = (ctypes.c_void_p * n)(*[_ptr(t) for t in bs])
    infos = (SolveInfo * n)()
    rc = lib().qcd_batch_solve(batch, xa, ba, _on_device(bs[0]), ctypes.byref(p), infos, _stream(stream))
    if raise_on_error and rc != QCD_OK:
        raise QcdError(rc, lib().qcd_batch_last_error(batch).decode())
    return rc, list(infos)

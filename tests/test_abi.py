"""Host-side checks of the C ABI: the library builds for sm_103a, loads and
exports every function include/qcd_gb300.h declares (no GPU calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcd_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qcd_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_10687_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("qcd_create", "qcd_set_gauge", "qcd_set_params", "qcd_build_clover", "qcd_apply_D",
                 "qcd_sap_apply", "qcd_solve", "qcd_grad", "qcd_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2109_10687_gb300 import binding
    assert sorted(binding.exported_symbols()) == declared_functions()


def test_version_string(lib):
    lib.qcd_version.restype = ctypes.c_char_p
    assert lib.qcd_version().decode().startswith("qcd_gb300")


def test_solve_defaults_match_header(lib):
    from paper_2109_10687_gb300 import binding
    binding._lib = None
    p = binding.qcd_solve_params_default()
    assert (p.tol, p.inner_tol, p.max_outer, p.max_inner, p.n_sap, p.n_jac) == (1e-10, 1e-6, 20, 500, 4, 4)
    assert (p.sap_prec, p.use_graph, p.x_is_guess, p.residual_prec, p.outer_restart) == (binding.PREC_SINGLE, 0, 0, 0, 0)


def test_solve_params_layout_matches_header():
    """The ctypes mirror of qcd_solve_params lists the header's fields in the
    header's order with the header's C types."""
    import re
    from paper_2109_10687_gb300 import binding
    text = open(HEADER).read()
    body = re.search(r"typedef struct qcd_solve_params \{(.*?)\} qcd_solve_params;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(double|int)\s+([A-Za-z0-9_]+)\s*;", body)
    ctypes_map = {"double": "c_double", "int": "c_int"}
    got = [(name, t.__name__) for name, t in binding.SolveParams._fields_]
    assert got == [(name, ctypes_map[t]) for t, name in fields]


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as C99 (no C++ or CUDA types in the ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "qcd_gb300.h"\n'
                   'int main(void) { qcd_solve_params p; qcd_solve_params_default(&p); return p.n_sap == 4 ? 0 : 1; }\n')
    res = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.dirname(HEADER), str(src)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr

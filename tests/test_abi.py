"""The C-ABI library loads and exports every symbol its header declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(omm_[A-Za-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    from paper_2209_05934_gb300 import omm
    return omm.lib()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("omm_create", "omm_set_HS", "omm_set_H", "omm_set_T", "omm_solve", "omm_solve_begin",
                 "omm_solve_progress", "omm_solve_end", "omm_batch_solve", "omm_md_guess", "omm_get_diag",
                 "omm_get_array", "omm_get_density", "omm_get_pattern", "omm_destroy", "omm_status_str",
                 "omm_op_dgemm", "omm_op_split_gemm", "omm_op_exact_gemm", "omm_op_quartic_coeffs",
                 "omm_op_quartic_coeffs_static", "omm_op_line_min", "omm_selftest_bounded_wait", "omm_op_convert"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    missing = [n for n in sorted(_declared()) if not hasattr(built, n)]
    assert not missing, missing


def test_status_strings(built):
    from paper_2209_05934_gb300 import omm
    assert omm.status_str(0) == "ok"
    assert "minimum" in omm.status_str(omm.ERR_LINESEARCH)
    assert omm.status_str(12345) == "unknown status"


def test_argument_errors_without_gpu(built):
    """Argument validation happens on the host, before any CUDA call."""
    import ctypes as C
    from paper_2209_05934_gb300 import omm
    h = C.c_void_p()
    assert built.omm_create(0, 1, 8, None, None, C.byref(h)) == omm.ERR_ARG
    assert built.omm_create(10, 11, 8, None, None, C.byref(h)) == omm.ERR_ARG
    assert built.omm_create(10, 2, 8, None, None, None) == omm.ERR_ARG
    assert built.omm_solve(None, None, 0, 1e-10, None, 0, None, None) == omm.ERR_ARG
    assert omm.op_dgemm(0, 0, -1, 2, 2, 1.0, None, 1, None, 1, 0.0, None, 1, None, 1) == omm.ERR_ARG
    assert omm.op_line_min(None, None, None) == omm.ERR_ARG
    assert built.omm_op_convert(7, 4, None, None, None, None) == omm.ERR_ARG
    assert built.omm_op_convert(0, 4, None, None, None, None) == omm.ERR_ARG


def test_options_reject_unknown_names(built):
    """Option names are checked against the C struct (a misspelt option must not pass silently)."""
    from paper_2209_05934_gb300 import omm
    o = omm.default_options(precon=-1, tau_T=5.0, split_digits=3)
    assert (o.precon, o.tau_T, o.split_digits, o.graphs) == (-1, 5.0, 3, 1)
    # the C defaults of the last fields land where the binding reads them (same layout)
    assert (o.screen_eps, o.gemm_pair, o.gemm_persistent, o.dir_digits) == (0.0, 1, 0, 1)
    with pytest.raises(TypeError):
        omm.default_options(precond=-1)

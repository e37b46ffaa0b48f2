"""The C ABI: the library builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here: these run without a GPU.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    with open(os.path.join(ROOT, "include", "mpr.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(mpr_[A-Za-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1710_03038_gb300 import build
    build.build()
    from paper_1710_03038_gb300 import _lib
    return _lib.load()


def test_header_declares_the_five_method_entry_points():
    names = _declared_functions()
    for n in ("mpr_init_grid", "mpr_estimate_T", "mpr_sweep", "mpr_energy", "mpr_predict"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1710_03038_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.EXPORTS)


def test_host_only_calls(lib):
    """Calls that touch no device: defaults, status strings, workspace sizing, argument errors."""
    import ctypes as C
    from paper_1710_03038_gb300 import _lib
    p = _lib.MprParams()
    assert lib.mpr_default_params(C.byref(p)) == 0
    assert (p.q, p.J, p.A_targ, p.k_a) == (0.5, 1.0, 0.3, 3.0)
    o = _lib.MprTOpts()
    assert lib.mpr_default_T_opts(C.byref(o)) == 0
    assert lib.mpr_status_string(0) == b"ok"
    Lx = _lib.int_array([64, 37])
    Ly = _lib.int_array([64, 53])
    nbytes = C.c_size_t()
    assert lib.mpr_workspace_size(2, Lx, Ly, None, 4, C.byref(p), None, C.byref(nbytes)) == 0
    worst = nbytes.value
    ng = _lib.i64_array([1000, 500])
    assert lib.mpr_workspace_size(2, Lx, Ly, ng, 4, C.byref(p), None, C.byref(nbytes)) == 0
    assert 0 < nbytes.value < worst
    # invalid arguments are rejected on the host
    bad = _lib.int_array([1, 37])
    assert lib.mpr_workspace_size(2, bad, Ly, None, 4, C.byref(p), None, C.byref(nbytes)) == 1
    assert lib.mpr_workspace_size(2, Lx, Ly, None, 0, C.byref(p), None, C.byref(nbytes)) == 1
    p.q = 0.7
    assert lib.mpr_workspace_size(2, Lx, Ly, None, 4, C.byref(p), None, C.byref(nbytes)) == 1
    assert b"q" in lib.mpr_last_error()
    out = C.c_void_p()
    p.q = 0.5
    # NULL inputs are rejected before any device work
    assert lib.mpr_init_grid(C.byref(out), 2, Lx, Ly, 4, C.byref(p), None, None, None, 0, None, 0,
                             None) == 1
    # cross-validated q: workspace sizing and argument checks, all before any device work
    qb = C.c_size_t()
    assert lib.mpr_select_q_workspace_size(64, 64, 8, C.byref(p), None, C.byref(qb)) == 0
    assert lib.mpr_workspace_size(1, _lib.int_array([64]), _lib.int_array([64]), None, 8,
                                  C.byref(p), None, C.byref(nbytes)) == 0
    assert qb.value > nbytes.value  # one context plus the staged inputs
    dummy = C.c_void_p(256)          # never dereferenced: the checks below fail first
    qs = (C.c_double * 2)(0.25, 0.6)
    sc = (C.c_double * 2)()
    assert lib.mpr_select_q(64, 64, dummy, dummy, dummy, 0, 2, qs, 8, 10, 10, C.byref(p), None,
                            dummy, qb, sc, None, None, None) == 1
    assert b"(0, 1/2]" in lib.mpr_last_error()
    qs[1] = 0.5
    assert lib.mpr_select_q(64, 64, dummy, dummy, dummy, 0, 2, qs, 8, 10, 0, C.byref(p), None,
                            dummy, qb, sc, None, None, None) == 1
    p.model = 1
    assert lib.mpr_select_q(64, 64, dummy, dummy, dummy, 0, 2, qs, 8, 10, 10, C.byref(p), None,
                            dummy, qb, sc, None, None, None) == 1
    assert b"MPR bond" in lib.mpr_last_error()
    p.model = 0


def test_no_cpu_fallback_in_product_package():
    """The package never imports the oracle (the CPU reference is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1710_03038_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, fn)) as f:
                    text = f.read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "mpr_oracle" not in text, fn

"""The C-ABI library loads and exports every entry point include/iobm.h declares
(no compute call: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "iobm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iobm_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1009_5300_gb300 import build_library, load
    build_library()
    return load()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("iobm_create", "iobm_solve", "iobm_transmission", "iobm_grad_V", "iobm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1009_5300_gb300._lib import SIGNATURES
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in SIGNATURES, f"binding lacks {name}"


def test_status_strings(lib):
    for code in range(0, 10):
        assert lib.iobm_status_string(code)


def test_default_options_and_binding_layout(lib):
    # the ctypes mirror of iobm_options matches the header's field list, and the
    # defaults documented beside iobm_default_options are what the library fills in
    import ctypes as C
    from paper_1009_5300_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "iobm.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} iobm_options;", src).group(1)
    fields = re.findall(r"\b(?:double|int)\s+([A-Za-z_0-9]+)\s*;", body)
    assert fields == [f for f, _ in _lib.Options._fields_]
    o = _lib.Options()
    lib.iobm_default_options(C.byref(o))
    assert (o.alpha, o.use_precond, o.tol, o.max_iter) == (1.8, _lib.IOBM_PRECOND_FOURIER, 1e-8, 20000)
    assert (o.precision, o.refine_delta, o.chunk) == (_lib.IOBM_MIXED, 0.01, 32)
    assert (o.max_iter_mixed, o.op_form, o.fp64_modes) == (1000, _lib.IOBM_OP_AUTO, -1)
    assert o.sigma_form == _lib.IOBM_SIGMA_FFT

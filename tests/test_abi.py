"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point
include/hisq.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hisq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hisq_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libhisq():
    from paper_2111_10354_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hisq_create", "hisq_destroy", "hisq_load_links", "hisq_dslash", "hisq_cg", "hisq_multishift_cg",
                 "hisq_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(libhisq):
    missing = [n for n in declared_functions() if not hasattr(libhisq, n)]
    assert not missing, missing


def test_error_strings_without_gpu(libhisq):
    libhisq.hisq_strerror.restype = ctypes.c_char_p
    assert libhisq.hisq_strerror(0) == b"success"
    assert libhisq.hisq_strerror(-6) == b"solver did not converge"
    assert libhisq.hisq_strerror(-99) == b"unknown error"


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2111_10354_gb300 as h
    monkeypatch.setattr(h, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(h, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        h.hisq_strerror(0)


def test_context_switches_reject_a_null_context_without_gpu(libhisq):
    """The per-context switches validate their context before anything else (no CUDA call is made)."""
    einval = -1
    for name in ("hisq_set_autotune", "hisq_set_pdl"):
        f = getattr(libhisq, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_int]
        assert f(None, 1) == einval, name

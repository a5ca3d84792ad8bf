"""The C ABI library (no GPU needed): it builds, loads, and exports every
entry point that include/gpufilter.h declares; the binding fails loudly when
the library is missing."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gpufilter.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(filter_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2212_09005_gb300 as gf

    return gf.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("filter_create", "filter_destroy", "filter_insert", "filter_query",
                 "filter_remove", "filter_count", "filter_get_stats", "filter_export"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    import paper_2212_09005_gb300 as gf

    assert sorted(gf.EXPORTS) == declared_functions()


def test_error_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.filter_error_string.restype = ctypes.c_char_p
    assert lib.filter_error_string(0) == b"ok"
    assert b"argument" in lib.filter_error_string(1)


def test_null_arguments_rejected_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    assert lib.filter_create(None, None, None) == 1
    assert lib.filter_insert(None, None, 0, None, None) == 1
    assert lib.filter_destroy(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2212_09005_gb300 as gf

    monkeypatch.setattr(gf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gf, "_lib", None)
    with pytest.raises(gf.FilterError):
        gf.lib()

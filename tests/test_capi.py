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
    assert lib.filter_insert_values(None, None, None, 0, None, None) == 1
    assert lib.filter_query_values(None, None, 0, None, None) == 1
    assert lib.filter_destroy(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2212_09005_gb300 as gf

    monkeypatch.setattr(gf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gf, "_lib", None)
    with pytest.raises(gf.FilterError):
        gf.lib()


def test_tcf_geometries_validated_without_gpu(libpath):
    """Block geometries are checked before any device memory is taken: the
    packed (f, B) pairs with kernels pass the check (and then fail only at the
    allocation on a machine without a GPU), the others are refused."""
    import paper_2212_09005_gb300 as gf

    lib = gf.lib()
    h = ctypes.c_void_p()

    def create(lg, f, mode=gf.MODE_BULK, v=0, B=0):
        return lib.filter_create(ctypes.byref(gf.FilterConfig(gf.FILTER_TCF, lg, f, mode, 1, 1, v, B)), None,
                                 ctypes.byref(h))

    ok_or_oom = (0, 2)
    for f, B in ((16, 8), (16, 32), (16, 64), (16, 128), (12, 21), (12, 0), (8, 64), (16, 16), (8, 32), (16, 0)):
        assert create(20, f, B=B) in ok_or_oom, (f, B)
    for f, B in ((16, 48), (16, 256), (12, 32), (8, 8), (10, 0)):
        assert create(20, f, B=B) == 1, (f, B)
    assert create(20, 16, mode=gf.MODE_POINT, B=64) == 1  # packed blocks: bulk mode only
    assert create(20, 12, mode=gf.MODE_POINT) == 1
    assert create(20, 16, v=4, B=64) == 1                  # no values
    assert create(7, 16, B=128) == 1                       # fewer than two blocks
    assert lib.filter_create(ctypes.byref(gf.FilterConfig(gf.FILTER_GQF, 12, 8, 0, 1, 1, 0, 16)), None,
                             ctypes.byref(h)) == 1


def test_group_configurations_rejected_without_gpu(libpath):
    """Group creation validates the member list before touching the device."""
    import paper_2212_09005_gb300 as gf

    lib = gf.lib()
    h = ctypes.c_void_p()

    def create(cfgs):
        arr = (gf.FilterConfig * len(cfgs))(*cfgs)
        return lib.filter_group_create(arr, len(cfgs), 1000, None, ctypes.byref(h))

    tcf = gf.FilterConfig(gf.FILTER_TCF, 12, 16, gf.MODE_BULK, 1, 1)
    gqf = gf.FilterConfig(gf.FILTER_GQF, 12, 8, 0, 1, 1)
    assert create([tcf, gqf]) == 1                                              # mixed kinds
    assert create([tcf, gf.FilterConfig(gf.FILTER_TCF, 12, 8, 0, 1, 1)]) == 1    # mixed tag widths
    assert create([gf.FilterConfig(gf.FILTER_TCF, 12, 16, gf.MODE_POINT, 1, 1)]) == 1  # point mode
    assert create([gf.FilterConfig(gf.FILTER_GQF, 40, 16, 0, 1, 1)]) == 1        # q + r beyond limits
    assert create([gf.FilterConfig(gf.FILTER_TCF, 12, 16, gf.MODE_BULK, 1, 1, 4)]) == 1  # members with values
    assert create([gf.FilterConfig(gf.FILTER_GQF, 12, 8, 0, 1, 1, 4)]) == 1      # GQF values: counters
    assert create([gf.FilterConfig(gf.FILTER_TCF, 12, 16, gf.MODE_BULK, 1, 1, 0, 64)]) == 1  # packed geometry
    assert create([gf.FilterConfig(gf.FILTER_TCF, 12, 12, gf.MODE_BULK, 1, 1)]) == 1  # 12-bit tags
    assert lib.filter_group_create(None, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.filter_group_insert(None, None, None, 0, None, None) == 1
    assert lib.filter_group_destroy(None) == 0


def test_server_arguments_rejected_without_gpu(libpath):
    import paper_2212_09005_gb300 as gf

    lib = gf.lib()
    h = ctypes.c_void_p()
    assert lib.filter_server_create(None, 0, 1, 16, ctypes.byref(h)) == 1
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.filter_server_create(arr, 1, 1, 16, ctypes.byref(h)) == 1  # null filter
    t = ctypes.c_uint64()
    assert lib.filter_server_submit(None, None, ctypes.byref(t)) == 1
    assert lib.filter_server_wait(None, 1, None, None) == 1
    assert lib.filter_server_destroy(None) == 0

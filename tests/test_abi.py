"""CPU-only checks of the C ABI: the library loads, exports every function declared in
include/isira.h, and rejects bad arguments before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def isira():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_07080_gb300 as m
    return m


def declared_functions():
    text = open(os.path.join(ROOT, "include", "isira.h")).read()
    return sorted(set(re.findall(r"ISIRA_API\s+[\w\s\*]+?\b(isira_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["isira_create", "isira_solve", "isira_eigpairs", "isira_get_stats", "isira_destroy",
                 "isira_error_string", "isira_default_opts"]:
        assert must in names


def test_library_exports_every_declared_symbol(isira):
    lib = C.CDLL(isira.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(declared_functions()) == sorted(isira.EXPORTED)


def test_struct_layouts_match_header(isira):
    text = open(os.path.join(ROOT, "include", "isira.h")).read()
    for struct, cls in [("isira_opts", isira.isira_opts), ("isira_stats", isira.isira_stats)]:
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)\s*(?:\[\s*\d+\s*\])?\s*[,;]", body)
        assert fields == [f for f, _ in cls._fields_], struct


def test_defaults_and_error_strings(isira):
    o = isira.default_opts()
    assert o.precision == isira.ISIRA_MIXED and o.tau_inner == 1e-3 and o.trim_index == -1
    for s in range(8):
        assert isira.lib.isira_error_string(s)
    assert b"unknown" in isira.lib.isira_error_string(99)


def test_invalid_arguments_are_rejected_without_a_gpu(isira):
    lib = isira.lib
    h = C.c_void_p()
    assert lib.isira_create(None, 10, 20, None, None, None, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_create(C.byref(h), 2, 2, 8, 8, None, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_create(C.byref(h), 10, 20, None, 8, None, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_solve(None, 3, 0.0, 1e-8, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_eigpairs(None, None, None, None, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_sym_eig(0, None, None, None, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_sym_eig(65, 8, 8, 8, None) == isira.ISIRA_ERR_INVALID_ARG
    lib.isira_destroy(None)

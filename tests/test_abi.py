"""The C ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares; oracle and product path stay independent.  No GPU needed."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(kk_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2103_11991_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_entry_points():
    names = _declared_functions()
    for n in ("kk_spgemm_handle_create", "kk_spgemm_symbolic", "kk_spgemm_numeric",
              "kk_spgemm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2103_11991_gb300 import spgemm
    assert set(_declared_functions()) <= set(spgemm.exported_symbols())


def test_status_strings_without_gpu(lib):
    lib.kk_status_string.restype = ctypes.c_char_p
    assert lib.kk_status_string(0) == b"KK_OK"
    assert lib.kk_status_string(5) == b"KK_ERR_CAPACITY"


def test_invalid_args_rejected_on_host(lib):
    # NULL handle pointers are rejected before any CUDA call
    assert lib.kk_spgemm_handle_create(None, None, None) == 1
    assert lib.kk_spgemm_destroy(None) == 1
    assert lib.kk_spgemm_options_default(None) == 1


def test_oracle_and_product_are_independent():
    pkg = os.path.join(ROOT, "paper_2103_11991_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
            assert "spgemm_oracle" not in txt, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2103_11991_gb300", txt, flags=re.M), f
            assert "kk_spgemm" not in txt and "csrc" not in txt, f


def _struct_fields(header, name):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r";", src)
    assert m, name
    return re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*;", m.group(1))


def test_binding_structs_match_header():
    # the ctypes mirrors of the option and matrix structs list the header's
    # fields in the header's order (all 32-bit or pointer fields)
    from paper_2103_11991_gb300 import spgemm as K
    assert [f for f, _ in K.KkOptions._fields_] == _struct_fields("kk_spgemm.h", "kk_spgemm_options")
    assert [f for f, _ in K.KkCsr._fields_] == _struct_fields("kk_spgemm.h", "kk_csr")


def test_options_default_fills_every_field(lib):
    from paper_2103_11991_gb300 import spgemm as K
    o = K.KkOptions()
    for f, _ in o._fields_:
        setattr(o, f, -12345)
    assert lib.kk_spgemm_options_default(ctypes.byref(o)) == 0
    assert all(getattr(o, f) != -12345 for f, _ in o._fields_)
    assert o.batched_learned == 0 and o.structure_cache == 1

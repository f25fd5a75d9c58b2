"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/*.h declares.
CPU only: no compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hadamag_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2601_07824_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("hadamag_sre", "hadamag_sre_mc", "hadamag_mana", "hadamag_sre_grad",
              "hadamag_sre_batched", "hadamag_create", "hadamag_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2601_07824_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_status_strings(lib):
    f = lib.hadamag_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ok"
    assert f(5) == b"device wait timed out"


def test_null_context_is_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    f = lib.hadamag_sre
    f.restype = ctypes.c_int
    assert f(None, None, 4, ctypes.c_double(2.0), 0, None, None, None) == 1
    g = lib.hadamag_create
    g.restype = ctypes.c_int
    assert g(None, 0) == 1

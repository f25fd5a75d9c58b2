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
    # the tuner controls and pins reject a null context (HADAMAG_ERR_INVALID_ARG) too
    for name, args in (("hadamag_set_autotune", (None, 1)),
                       ("hadamag_set_grad_xbatch", (None, 17, 2)),
                       ("hadamag_set_twopass_shape", (None, 18, ctypes.c_double(2.0), 2, 2, 0, 1))):
        h = getattr(lib, name)
        h.restype = ctypes.c_int
        assert h(*args) == 1, name


def test_typed_binding_marshals_every_argument_without_gpu():
    # the binding's argtypes convert each Python argument; a null context returns
    # INVALID_ARG before any CUDA call
    import ctypes as C

    from paper_2601_07824_gb300 import _lib
    lib = _lib.load()
    M, means = C.c_double(), (C.c_double * 4)()
    assert lib.hadamag_sre_ti(None, None, 10, 4, 100, 10, C.c_uint64(2 ** 64 - 1), 0.0, 1, 0, C.byref(M), C.byref(M),
                              means, None, None) == 1
    assert lib.hadamag_sre_even_sector(None, None, 10, 2.0, 0, C.byref(M), C.byref(M), None) == 1
    assert lib.hadamag_mana_mixed(None, None, 4, 0, C.byref(M), means, None) == 1
    assert lib.hadamag_reduced_density_matrix(None, None, 4, 0, (C.c_int * 2)(0, 1), 2, None, None) == 1
    assert lib.hadamag_sre_mc(None, None, 10, 100, C.c_uint64(5), 0, C.byref(M), C.byref(M), None) == 1
    assert lib.hadamag_sre_terms(None, None, 10, 2.0, 0, None, 4, None, None) == 1

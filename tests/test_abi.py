"""The C-ABI library builds, loads and exports every entry point include/ts.h declares (no GPU
needed: nothing here launches device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    with open(os.path.join(ROOT, "include", "ts.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ts_build_index", "ts_search", "ts_free", "ts_last_error",
                     "ts_result_count", "ts_result_arrays"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1410_2698_gb300 import _lib
    lib = _lib.load()
    cdll = ctypes.CDLL(_lib.lib_path())
    for name in _declared_functions():
        assert hasattr(cdll, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert lib.ts_version().decode().startswith("ts_gb300")


def test_binding_has_no_fallback():
    # the binding only marshals: every public function goes through the loaded library
    import paper_1410_2698_gb300.api as api
    src = open(api.__file__).read()
    assert "oracle" not in src
    assert "import torch" in src  # device memory / streams only


def test_errors_are_reported_without_a_gpu():
    # argument validation happens before any device work
    from paper_1410_2698_gb300 import _lib
    lib = _lib.load()
    out = ctypes.c_void_p()
    st = lib.ts_build_index(None, None, None, ctypes.byref(out))
    assert st == 1
    assert "NULL" in lib.ts_last_error().decode()
    lib.ts_free(None)

"""The C ABI library builds, loads and exports every entry point declared in
include/extconv.h (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "extconv.h")).read()
    return sorted(set(re.findall(r"\b(ext_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    from paper_2006_13188_gb300 import EXPORTED
    assert sorted(EXPORTED) == declared_symbols()


def test_library_exports_every_declared_symbol():
    from paper_2006_13188_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    from paper_2006_13188_gb300 import lib
    L = lib()
    assert L.ext_status_string(0) == b"EXT_OK"
    assert L.ext_status_string(2) == b"EXT_ERR_UNSUPPORTED"

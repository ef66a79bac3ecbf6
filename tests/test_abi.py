"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/*.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2311_02206_gb300 import build as hisa_build
from paper_2311_02206_gb300 import hisa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**(hisa_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = hisa_build.build()
    return ctypes.CDLL(path)


def test_headers_declare_entry_points():
    names = declared_functions()
    assert {"hisa_create", "hisa_run", "hisa_read_relation", "hisa_sort_codes", "hisa_join_codes"} <= names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert declared_functions() == set(hisa.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.hisa_status_string.restype = ctypes.c_char_p
    assert lib.hisa_status_string(0) == b"ok"
    assert lib.hisa_status_string(-5) == b"device-side wait timed out"


def test_config_default(lib):
    cfg = hisa.Config()
    assert hisa.load_library().hisa_config_default(ctypes.byref(cfg)) == 0
    assert abs(cfg.load_factor - 0.8) < 1e-6 and cfg.ebm_k == 2.0 and cfg.device == -1

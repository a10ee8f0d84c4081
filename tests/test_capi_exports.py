"""The C ABI library loads and exports every function include/slim.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1912_07962_gb300 import build, slim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "slim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(slim_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declarations_match_binding():
    assert _declared() == sorted(slim.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_loads_library():
    assert slim.load() is not None


def test_null_arguments_are_rejected_without_a_gpu(lib):
    lib.slim_create.restype = ctypes.c_int
    assert lib.slim_create(None, None, 0, ctypes.c_double(1.0), None, None) == slim.SLIM_EINVAL
    lib.slim_last_error.restype = ctypes.c_char_p
    lib.slim_last_error.argtypes = [ctypes.c_void_p]
    assert lib.slim_last_error(None) == b"null context"

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
    return sorted(set(re.findall(r"\b(slim_[a-z0-9_]+)\s*\(", src)))


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


def test_layer_entry_points_reject_bad_arguments_without_a_gpu(lib):
    # validation happens before any CUDA call
    VP, I = ctypes.c_void_p, ctypes.c_int
    f = lib.slim_unet_conv3x3
    f.argtypes = [VP, I, I, I, I, VP, VP, I, I, VP, VP]
    f.restype = I
    dummy = VP(16)
    assert f(None, 1, 1, 8, 8, dummy, None, 1, 0, dummy, None) == slim.SLIM_EINVAL
    assert f(dummy, 0, 1, 8, 8, dummy, None, 1, 0, dummy, None) == slim.SLIM_EINVAL
    assert f(dummy, 1, 1, 8, 8, dummy, None, 70000, 0, dummy, None) == slim.SLIM_EINVAL
    assert f(dummy, 1 << 14, 1, 256, 256, dummy, None, 1, 0, dummy, None) == slim.SLIM_EINVAL
    g = lib.slim_unet_tconv2x2_grad
    g.argtypes = [VP, VP, I, I, I, I, VP, I, VP, VP, VP, VP]
    g.restype = I
    assert g(dummy, dummy, 1, 1, 8, 8, dummy, 1, None, None, None, None) == slim.SLIM_EINVAL

"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/taps.h declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "taps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(
        r"^\s*(?:const\s+)?(?:int|void|char|double|long long)\s*\*?\s*(taps_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2503_13933_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("taps_assemble_1d", "taps_sweep", "taps_solve", "taps_eval_grid",
                     "taps_eval_points", "taps_problem_create", "taps_residual"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2503_13933_gb300 import taps
    assert sorted(taps.SIGNATURES) == _declared()


def test_status_strings_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.taps_status_string.restype = ctypes.c_char_p
    assert L.taps_status_string(0) == b"ok"
    assert b"singular" in L.taps_status_string(-2)

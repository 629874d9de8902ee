"""The bounds-checked variant of the library (-DCVWENO_CHECK) builds and exports every
entry point that include/cvweno.h declares, like the normal library (no compute calls:
this runs without a GPU)."""
import ctypes

import pytest

from tests.test_abi import declared_functions


@pytest.fixture(scope="module")
def checked_lib():
    from paper_2601_16911_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libcvweno_check.so")
    return ctypes.CDLL(path)


def test_checked_library_exports_every_declared_symbol(checked_lib):
    missing = [n for n in declared_functions() if not hasattr(checked_lib, n)]
    assert not missing, missing


def test_check_extents_argument_errors_without_gpu(checked_lib):
    f = checked_lib.cvweno_mesh_set_check_extents
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
    assert f(None, 10, 10) == 1  # CVWENO_ERR_ARG: no mesh
    checked_lib.cvweno_status_string.restype = ctypes.c_char_p
    assert b"bounds check" in checked_lib.cvweno_status_string(8)

"""The C ABI library loads and exports every entry point that include/cvweno.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cvweno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cvweno_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_16911_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("cvweno_mesh_create", "cvweno_sensor", "cvweno_residual", "cvweno_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2601_16911_gb300 import cvweno
    declared = set(declared_functions())
    assert declared == set(cvweno.exported_symbols())
    for n in declared:
        assert callable(getattr(cvweno, n)), n


def test_status_strings_and_argument_errors_without_gpu(lib):
    lib.cvweno_status_string.restype = ctypes.c_char_p
    assert lib.cvweno_status_string(0) == b"ok"
    assert lib.cvweno_status_string(6) == b"unsupported configuration"
    # NULL arguments are rejected on the host, before any CUDA call
    lib.cvweno_mesh_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.cvweno_mesh_create(None, None) == 1
    lib.cvweno_sensor.argtypes = [ctypes.c_void_p] * 5
    assert lib.cvweno_sensor(None, None, None, None, None) == 1

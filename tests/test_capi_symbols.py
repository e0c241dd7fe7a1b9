"""The C-ABI library builds, loads without a GPU, and exports every symbol of include/firal.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_07392_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "firal.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const char\*|int32_t|int64_t)\s+(firal_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported(lib):
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_declares_every_symbol():
    from paper_2409_07392_gb300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == header_symbols()


def test_status_strings_and_build_info(lib):
    lib.firal_status_string.restype = ctypes.c_char_p
    assert lib.firal_status_string(0) == b"FIRAL_OK"
    assert lib.firal_status_string(-3) == b"FIRAL_ERR_NOT_SPD"
    assert lib.firal_build_info() & 1


def test_struct_layouts_match_header():
    from paper_2409_07392_gb300 import _lib as L
    assert ctypes.sizeof(L.FiralPool) == 40
    assert ctypes.sizeof(L.FiralCGOpts) == 16
    assert ctypes.sizeof(L.FiralRelaxOpts) == 56
    assert L.FiralRelaxOpts.beta0.offset == 24 and L.FiralRelaxOpts.md_tol.offset == 48
    assert ctypes.sizeof(L.FiralStepStats) == 48


def test_null_arguments_rejected_without_gpu(lib):
    lib.firal_problem_destroy.argtypes = [ctypes.c_void_p]
    assert lib.firal_problem_destroy(None) == 0
    lib.firal_destroy.argtypes = [ctypes.c_void_p]
    assert lib.firal_destroy(None) == 0

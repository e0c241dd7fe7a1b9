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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors agree with the C compiler's layout of include/firal.h."""
    import shutil
    import subprocess
    from paper_2409_07392_gb300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = {
        "sizeof(firal_pool)": ctypes.sizeof(L.FiralPool),
        "sizeof(firal_hess0)": ctypes.sizeof(L.FiralHess0),
        "sizeof(firal_cg_opts)": ctypes.sizeof(L.FiralCGOpts),
        "offsetof(firal_cg_opts, block)": L.FiralCGOpts.block.offset,
        "sizeof(firal_relax_opts)": ctypes.sizeof(L.FiralRelaxOpts),
        "offsetof(firal_relax_opts, cg)": L.FiralRelaxOpts.cg.offset,
        "offsetof(firal_relax_opts, beta0)": L.FiralRelaxOpts.beta0.offset,
        "offsetof(firal_relax_opts, seed)": L.FiralRelaxOpts.seed.offset,
        "offsetof(firal_relax_opts, md_tol)": L.FiralRelaxOpts.md_tol.offset,
        "sizeof(firal_step_stats)": ctypes.sizeof(L.FiralStepStats),
        "sizeof(firal_round_opts)": ctypes.sizeof(L.FiralRoundOpts),
        "sizeof(firal_al_opts)": ctypes.sizeof(L.FiralAlOpts),
        "offsetof(firal_al_opts, relax)": L.FiralAlOpts.relax.offset,
        "offsetof(firal_al_opts, eta)": L.FiralAlOpts.eta.offset,
    }
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", (size_t)({k}));\n' for k in checks)
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"firal.h\"\n"
                   "int main(void) {\n" + body + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in got] == list(checks.values()), dict(zip(checks, got))


def test_null_arguments_rejected_without_gpu(lib):
    lib.firal_problem_destroy.argtypes = [ctypes.c_void_p]
    assert lib.firal_problem_destroy(None) == 0
    lib.firal_destroy.argtypes = [ctypes.c_void_p]
    assert lib.firal_destroy(None) == 0


def test_block_cache_entry_points_without_gpu(lib):
    lib.firal_cache_bytes.restype = ctypes.c_int64
    assert lib.firal_cache_bytes() == 0
    assert lib.firal_cache_trim() == 0

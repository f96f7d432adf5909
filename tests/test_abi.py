"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, and exports every
function that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_00541_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hec_from_csr", "sptrsv_analyze", "sptrsv_lower", "sptrsv_upper", "ilu_apply", "spmv",
                     "fgmres_solve", "ilu_factor", "hec_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_has_no_torch_dependency(lib):
    # the boundary is plain C: the shared object must not link against torch
    path = os.path.join(ROOT, "paper_1606_00541_gb300", "libhec.so")
    import subprocess
    out = subprocess.run(["ldd", path], capture_output=True, text=True).stdout
    assert "torch" not in out and "c10" not in out


def test_version_and_counter_without_gpu(lib):
    lib.hec_version.restype = ctypes.c_int
    lib.hec_launch_count.restype = ctypes.c_longlong
    assert lib.hec_version() >= 1
    assert lib.hec_launch_count() >= 0


def test_invalid_arguments_rejected_on_host(lib):
    # argument checks happen before any device work, so they run without a GPU
    lib.sptrsv_analyze.restype = ctypes.c_int
    out = ctypes.c_void_p()
    st = lib.sptrsv_analyze(ctypes.c_int(-1), None, None, ctypes.c_int(0), ctypes.byref(out), None)
    assert st == 1  # HEC_ERR_INVALID_ARG
    lib.hec_last_error.restype = ctypes.c_char_p
    assert b"bad argument" in lib.hec_last_error()
    st = lib.sptrsv_analyze(ctypes.c_int(4), None, None, ctypes.c_int(2), ctypes.byref(out), None)
    assert st == 1
    lib.fgmres_solve.restype = ctypes.c_int
    st = lib.fgmres_solve(None, None, 1, None, 1, None, 1, 30, ctypes.c_double(1e-8), 10, None, None)
    assert st == 1


def test_binding_fails_loudly_without_the_library():
    """The Python binding has no CPU fallback: loaded from a place without libhec.so it raises
    ImportError instead of defining the calls."""
    import types
    src_path = os.path.join(ROOT, "paper_1606_00541_gb300", "hec.py")
    mod = types.ModuleType("hec_without_library")
    mod.__file__ = os.path.join(ROOT, "no_such_directory", "hec.py")
    with pytest.raises(ImportError, match="libhec.so is not built"):
        exec(compile(open(src_path).read(), mod.__file__, "exec"), mod.__dict__)
    assert "ilu_apply" not in mod.__dict__


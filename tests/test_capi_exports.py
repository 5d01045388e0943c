"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/bh.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bh_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2005_00281_gb300.build import build_library
    return build_library()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("bh_model_create", "bh_forward", "bh_residual_misfit", "bh_adjoint_gradient",
              "bh_precondition", "bh_update"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2005_00281_gb300.bh import EXPORTS
    assert set(EXPORTS) == declared_symbols()


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.bh_status_string.restype = ctypes.c_char_p
    lib.bh_status_string.argtypes = [ctypes.c_int]
    assert lib.bh_status_string(0) == b"ok"
    assert lib.bh_status_string(2) == b"CFL condition violated"

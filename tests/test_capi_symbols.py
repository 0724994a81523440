"""The C-ABI library loads and exports every entry point include/nemd.h declares.

No compute calls: this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_3784_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(nemd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nemd_set_flow", "nemd_set_state", "nemd_build_cells", "nemd_compute_forces"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1412_3784_gb300 import nemd
    assert set(nemd.EXPORTED) == set(declared_functions())
    for n in nemd.EXPORTED:
        assert callable(getattr(nemd, n))


def test_null_arguments_rejected_without_gpu(lib):
    # argument checks happen before any CUDA call
    lib.nemd_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.nemd_create(None, 0, None) == 1
    lib.nemd_set_flow.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_double]
    assert lib.nemd_set_flow(None, None, None, None, 1.0) == 1
    lib.nemd_last_error.restype = ctypes.c_char_p
    lib.nemd_last_error.argtypes = [ctypes.c_void_p]
    assert lib.nemd_last_error(None) == b"null context"

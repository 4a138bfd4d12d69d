"""CPU checks of the C-ABI library: it builds, loads, and exports every
function include/ljmd.h declares.  No compute calls (no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2406_04210_gb300 import build, ljmd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    try:
        path = build.build()
    except RuntimeError as e:   # no nvcc: nothing to check
        pytest.skip(str(e))
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"md_box_create", "md_set_lj", "md_neighbour_update", "md_force", "md_integrate",
            "md_adjoint"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    assert set(ljmd.EXPORTS) == _declared()


def test_status_strings(lib):
    lib.md_status_string.restype = ctypes.c_char_p
    for s in range(9):
        assert lib.md_status_string(s)


def test_bad_arguments_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.md_batch_create(ctypes.byref(h), 0, None, None, None, None, None, 0, None) == 1
    assert lib.md_box_destroy(None) == 1
    # option setters and getters refuse a missing box
    k = ctypes.c_int32()
    for setter in ("md_set_force_kernel", "md_set_list_kernel", "md_set_graph_conditional"):
        assert getattr(lib, setter)(None, 0) == 1, setter
    for getter in ("md_get_force_kernel", "md_get_list_kernel", "md_get_graph_conditional"):
        assert getattr(lib, getter)(None, ctypes.byref(k)) == 1, getter

"""The C-ABI library loads and exports every function that include/ssa.h declares (no GPU needed:
no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ssa_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2602_19775_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_expected_entry_points():
    from paper_2602_19775_gb300._lib import EXPORTS
    assert _declared() == set(EXPORTS)


def test_library_exports_every_declared_symbol(built_lib):
    for name in _declared():
        assert hasattr(built_lib, name), name


def test_binding_declares_signatures_without_gpu():
    from paper_2602_19775_gb300 import _lib
    lib = _lib.lib()
    assert lib.ssa_last_error() is not None
    # argument errors are reported without touching a device
    h = ctypes.c_void_p()
    st = lib.ssa_create_network(0, 1, None, None, None, None, 1, None, ctypes.byref(h))
    assert st == -1 and b"n_species" in lib.ssa_last_error()
    assert lib.ssa_forward_workspace_bytes(None, 1, 1, None) == 0

"""The C-ABI library loads and exports every symbol include/snap.h declares (CPU only,
no compute calls), and the Python binding fails loudly when the library is missing."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1111_5572_gb300 as snap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(snap_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    assert os.path.exists(snap.LIB_PATH)
    return snap.LIB_PATH


def test_library_exports_every_declared_symbol(lib_path):
    declared = _declared()
    assert "snap_index_build" in declared and "snap_align" in declared
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert hasattr(lib, name), name
    assert set(snap.EXPORTS) <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (snap_[a-z_0-9]+)", out))
    assert declared <= exported


def test_invalid_arguments_fail_without_a_gpu(lib_path):
    lib = snap.load_library()
    h = ctypes.c_void_p()
    # argument checks happen before any CUDA call
    assert lib.snap_index_build(None, 100, 20, ctypes.byref(h)) == snap.SNAP_E_INVAL
    assert b"NULL" in lib.snap_last_error()
    g = (ctypes.c_uint8 * 100)()
    assert lib.snap_index_build(g, 100, 7, ctypes.byref(h)) == snap.SNAP_E_INVAL
    assert lib.snap_index_build(g, 100, 33, ctypes.byref(h)) == snap.SNAP_E_INVAL
    assert lib.snap_index_build(g, 10, 20, ctypes.byref(h)) == snap.SNAP_E_INVAL
    assert lib.snap_server_destroy(None) == snap.SNAP_OK
    assert lib.snap_index_free(None) == snap.SNAP_OK


def test_missing_library_raises(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        snap._lib = None
        try:
            snap.load_library(str(tmp_path / "nope.so"))
        finally:
            snap._lib = None

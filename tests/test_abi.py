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


def test_struct_layouts_match_the_header(tmp_path):
    # the binding's ctypes structures against the C compiler's layout of include/snap.h:
    # every field at the same offset, every struct the same size
    structs = {"snap_params": snap.snap_params, "snap_result": None,
               "snap_index_info": snap.snap_index_info, "snap_call_stats": snap.snap_call_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "snap.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        fields = ([f for f in snap.RESULT_DTYPE.names if f != "pad"] if cls is None
                  else [f for f, _ in cls._fields_])
        for field in fields:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for name, cls in structs.items():
        if cls is None:
            assert int(out[f"{name} size"]) == snap.RESULT_DTYPE.itemsize
            for field in snap.RESULT_DTYPE.names:
                if field != "pad":
                    assert int(out[f"{name}.{field}"]) == snap.RESULT_DTYPE.fields[field][1]
            continue
        assert int(out[f"{name} size"]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(out[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)

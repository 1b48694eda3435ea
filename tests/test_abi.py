"""The C-ABI library loads and exports every function include/bst.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_]+)\s*\(", txt)) - {"sizeof"})


@pytest.fixture(scope="module")
def lib():
    from paper_1704_08364_gb300 import build
    build.build_lib("bst")
    return ctypes.CDLL(os.path.join(ROOT, "paper_1704_08364_gb300", "libbst.so"))


def test_exports_every_declared_symbol(lib):
    names = _declared("bst.h")
    assert "bst_fbp" in names and "radon_adjoint" in names and "brute_backproject" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header():
    from paper_1704_08364_gb300 import _lib
    assert set(_declared("bst.h")) == set(_lib.SIGNATURES)


def test_status_strings(lib):
    f = lib.bst_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ok"
    assert b"workspace" in f(3)


def test_invalid_arguments_need_no_device(lib):
    from paper_1704_08364_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    th = (ctypes.c_float * 4)(0.0, 0.5, 0.4, 1.0)          # not increasing
    assert L.bst_plan_create(ctypes.byref(h), 16, 4, th, 2) == 1 and not h.value
    th = (ctypes.c_float * 4)(0.0, 0.5, 1.0, 3.2)          # >= pi
    assert L.bst_plan_create(ctypes.byref(h), 16, 4, th, 2) == 1
    th = (ctypes.c_float * 4)(0.0, 0.5, 1.0, 1.5)
    assert L.bst_plan_create(ctypes.byref(h), 15, 4, th, 2) == 2   # odd N
    assert L.bst_plan_create(ctypes.byref(h), 2500, 4, th, 2) == 2  # M = 5000
    assert L.bst_plan_create(ctypes.byref(h), 16, 4, th, 3) == 2   # pad factor
    assert L.bst_plan_create(None, 16, 4, th, 2) == 1
    assert L.bst_fbp(None, None, 1, None, None, None, 0, None) == 1
    assert L.bst_workspace_bytes(None, 4) == 0
    assert L.bst_plan_set_gridding(None, 1, 6) == 1
    assert L.bst_fbp_backward(None, None, None, 1, None, None, None, None, 0, None) == 1
    k, w = ctypes.c_int(0), ctypes.c_int(0)
    assert L.bst_plan_get_gridding(None, ctypes.byref(k), ctypes.byref(w)) == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No fallback: the binding raises when the compiled library is absent."""
    from paper_1704_08364_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(str(tmp_path / "libbst.so"))


def test_forward_config_struct_matches_the_binding(tmp_path):
    """bst_fwd_config_t as the C compiler lays it out (size, and the offset of
    each field in header order) equals the binding's ctypes structure, so a
    field added to one side without the other fails here, not in a GPU call."""
    import shutil
    import subprocess
    from paper_1704_08364_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    txt = open(os.path.join(ROOT, "include", "bst.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} bst_fwd_config_t;", txt, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\bint\s+(\w+)\s*;", body)
    assert fields == [f for f, _ in _lib.FwdConfig._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n"
                   "typedef struct {" + body + "} cfg_t;\n"
                   "int main(void) { printf(\"%zu\", sizeof(cfg_t));"
                   + "".join(f' printf(" %zu", offsetof(cfg_t, {f}));' for f in fields)
                   + " printf(\"\\n\"); return 0; }\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", str(src), "-o", str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.split()]
    want = [ctypes.sizeof(_lib.FwdConfig)] + [getattr(_lib.FwdConfig, f).offset for f in fields]
    assert got == want

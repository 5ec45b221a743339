"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/hm.h; the Python binding covers the same
names. No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2602_22976_gb300 as hmlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^[A-Za-z_][\w\s\*]*?\b(hm_\w+)\s*\(", text, flags=re.M)


@pytest.fixture(scope="module")
def libpath():
    return hmlib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    assert len(names) == len(set(names))
    assert set(names) == set(hmlib.ENTRY_POINTS)
    for core in ("hm_create", "hm_match", "hm_result", "hm_destroy", "hm_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hm_\w+)$", out, flags=re.M))
    missing = set(declared_functions()) - exported
    assert not missing, f"not exported: {missing}"


def test_library_loads_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(L, name)
    L.hm_last_error.restype = ctypes.c_char_p
    assert L.hm_last_error() == b""
    # argument checks that run before any CUDA call
    h = ctypes.c_void_p()
    L.hm_create.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                            ctypes.c_void_p]
    assert L.hm_create(ctypes.byref(h), -1, 0, None, None, None, 0, 0, None) == hmlib.HM_EINVAL
    assert b"n must be" in L.hm_last_error()
    assert L.hm_create(None, 1, 1, None, None, None, 0, 0, None) == hmlib.HM_EINVAL
    assert L.hm_create(ctypes.byref(h), 1, 1, None, None, None, 0, 0x80, None) == hmlib.HM_EINVAL
    L.hm_set_round_cap.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert L.hm_set_round_cap(None, 5) == hmlib.HM_EINVAL
    L.hm_destroy.argtypes = [ctypes.c_void_p]
    L.hm_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(hmlib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hmlib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        hmlib.lib()


def test_build_targets_sm103a_only():
    import importlib
    b = importlib.import_module("paper_2602_22976_gb300.build")
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]

"""The C-ABI library loads and exports every entry point that include/wpcd.h
declares (no device needed), and the binding's list matches the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(wpcd_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2106_00454_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    d = _declared()
    for name in ["wpcd_mesh", "wpcd_project", "wpcd_diag", "wpcd_tmatrix", "wpcd_observables", "wpcd_solve"]:
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_list_matches_header():
    from paper_2106_00454_gb300 import _lib
    assert set(_lib.EXPORTED) == _declared()


def test_strerror_without_device(lib):
    f = lib.wpcd_strerror
    f.restype = ctypes.c_char_p
    assert f(0) == b"ok"
    assert b"budget" in f(-3)


def test_create_rejects_bad_arguments_without_device(lib):
    f = lib.wpcd_create
    f.restype = ctypes.c_int
    assert f(None, 0, 0, None) == -1   # null out pointer
    h = ctypes.c_void_p()
    assert f(ctypes.byref(h), -1, 0, None) == -1  # bad device


def test_null_context_is_rejected_without_device(lib):
    """Every entry point that takes a context returns WPCD_ERR_ARG (or a zero
    count) for a null one, before touching the device."""
    from paper_2106_00454_gb300 import _lib
    skip = {"wpcd_create", "wpcd_strerror", "wpcd_channel_solve_noalloc", "wpcd_destroy", "wpcd_release_result"}
    zero_ok = {"wpcd_kernel_launches", "wpcd_bytes_in_use", "wpcd_tuning"}
    checked = 0
    for name, (res, argtypes) in _lib._SIG.items():
        if name in skip or not argtypes or argtypes[0] is not ctypes.c_void_p:
            continue
        f = getattr(lib, name)
        f.restype, f.argtypes = res, argtypes
        args = [t() if t is not ctypes.c_void_p and not isinstance(t, type(ctypes.POINTER(ctypes.c_int)))
                else None for t in argtypes]
        got = f(*args)
        if name in zero_ok:
            assert got == 0, name
        else:
            assert got == -1, (name, got)
        checked += 1
    assert checked >= 25


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the compiled library absent the binding raises instead
    of computing anything another way (the product path has no CPU route)."""
    from paper_2106_00454_gb300 import _lib, api
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libwpcd.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()
    with pytest.raises(RuntimeError, match="missing"):
        api.Context(0)

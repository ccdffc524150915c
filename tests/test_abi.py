"""The C ABI library builds for sm_103a, loads, and exports every function that
include/pmmm.h declares; the binding refuses to run without it (no fallback).
No CUDA compute is called here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pmmm.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1409_5981_gb300 as pk
    from paper_1409_5981_gb300 import buildlib as b
    path = b.build()
    assert os.path.exists(path)
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "pmmm_compute" in names and "pmmm_plan_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_abi():
    import paper_1409_5981_gb300 as pk
    assert set(_declared()) == set(pk._SIGS)


def test_host_only_calls(lib):
    lib.pmmm_strerror.restype = ctypes.c_char_p
    lib.pmmm_strerror.argtypes = [ctypes.c_int]
    assert lib.pmmm_strerror(0) == b"ok"
    assert lib.pmmm_strerror(-3).startswith(b"particle outside")
    lib.pmmm_abi_version.restype = ctypes.c_int
    assert lib.pmmm_abi_version() == 1
    import paper_1409_5981_gb300 as pk
    c = pk._Config()
    pk._lib().pmmm_config_init(ctypes.byref(c))
    assert c.p == 4 and c.cutoff == 1 and c.sign == 1.0 and list(c.mesh) == [8, 8, 8]
    # invalid configurations are rejected before any device call
    h = ctypes.c_void_p()
    c.p = 99
    assert pk._lib().pmmm_plan_create(ctypes.byref(c), None, ctypes.byref(h)) == pk.ERR_UNSUPPORTED
    c.p = 4
    c.mesh[0] = 6
    assert pk._lib().pmmm_plan_create(ctypes.byref(c), None, ctypes.byref(h)) == pk.ERR_UNSUPPORTED
    c.mesh[0] = 8
    c.box_len[1] = -1.0
    assert pk._lib().pmmm_plan_create(ctypes.byref(c), None, ctypes.byref(h)) == pk.ERR_INVALID_ARG
    c.box_len[1] = 1.0
    c.boundary, c.mesh[2] = pk.PERIODIC, 2
    assert pk._lib().pmmm_plan_create(ctypes.byref(c), None, ctypes.byref(h)) == pk.ERR_UNSUPPORTED
    assert h.value is None


def test_no_fallback_without_library(tmp_path, monkeypatch):
    import paper_1409_5981_gb300 as pk
    monkeypatch.setattr(pk, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pk, "_LIB", None)
    with pytest.raises(RuntimeError, match="missing"):
        pk._lib()

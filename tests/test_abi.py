"""The C ABI library builds for sm_103a, loads, and exports every symbol include/coop.h declares.

CPU-only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

import pytest

import paper_1707_01989_gb300 as coop
from paper_1707_01989_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(coop_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared("coop.h")
    for required in ["coop_init", "coop_bfs", "coop_sssp", "coop_request_resources", "coop_release"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = coop.load_library()
    for name in _declared("coop.h"):
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_library_targets_sm103a_only():
    cmd = _build.build_command("x.so")
    assert "arch=compute_103a,code=sm_103a" in cmd
    assert sum("arch=" in c for c in cmd) == 1


def test_status_strings():
    assert coop.coop_status_string(0) == "COOP_OK"
    assert coop.coop_status_string(-4) == "COOP_ETIMEOUT"
    assert coop.coop_status_string(-7) == "COOP_EGRAPH"


def test_bad_arguments_are_rejected_without_a_gpu():
    lib = coop.load_library()
    # null context / null out pointers are refused before any CUDA call
    assert lib.coop_init(0, 0, 0, None) == coop.COOP_EINVAL
    assert lib.coop_init(0, -1, 0, ctypes.byref(ctypes.c_void_p())) == coop.COOP_EINVAL
    assert lib.coop_init(0, 0, 77, ctypes.byref(ctypes.c_void_p())) == coop.COOP_EINVAL
    assert lib.coop_bfs(None, None, 0, None, None, None) == coop.COOP_EINVAL
    assert lib.coop_release(None, 1) == coop.COOP_EINVAL
    assert lib.coop_request_resources(None, 1, 0, None) == coop.COOP_EINVAL
    assert lib.coop_saxpy(0, 10, 1.0, None, None, None) == coop.COOP_EINVAL
    assert lib.coop_destroy(None) == coop.COOP_OK


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    """The binding raises CoopUnavailable instead of computing anything on the host."""
    import importlib
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_build, "build_library", lambda *a, **k: (_ for _ in ()).throw(RuntimeError("no nvcc")))
    monkeypatch.setattr(coop, "_lib", None)
    with pytest.raises(coop.CoopUnavailable):
        coop.load_library()

"""The C ABI library loads and exports every entry point declared in include/lmdg.h (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lmdg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lmdg_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_01027_gb300 import buildlib
    if not os.path.exists(buildlib.LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build liblmdg")
        buildlib.build()
    return ctypes.CDLL(buildlib.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"lmdg_setup", "lmdg_sweep", "lmdg_solve", "lmdg_adjoint", "lmdg_destroy", "lmdg_strerror"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_host_only_entry_points(lib):
    lib.lmdg_strerror.restype = ctypes.c_char_p
    assert b"spin limit" in lib.lmdg_strerror(-6)
    from paper_1907_01027_gb300.lmdg import Options
    o = Options()
    assert lib.lmdg_default_options(ctypes.byref(o)) == 0
    assert o.restart == 30 and abs(o.tol - 1e-8) < 1e-20 and o.precond == 1
    assert lib.lmdg_default_options(None) == -1


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    from paper_1907_01027_gb300 import lmdg, buildlib
    monkeypatch.setattr(buildlib, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lmdg, "_LIB", None)
    with pytest.raises(ImportError):
        lmdg._lib()

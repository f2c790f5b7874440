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


def test_binding_layouts_match_header(tmp_path):
    """The ctypes structures and constants of the binding agree with include/lmdg.h: field offsets and sizes of
    every struct and the values of the enums, from a C program compiled against the header."""
    import subprocess
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1907_01027_gb300 import lmdg as L
    structs = {"lmdg_options": L.Options, "lmdg_stats": L.Stats, "lmdg_mesh": L.Mesh, "lmdg_quadrature": L.Quad}
    consts = {"LMDG_STD": L.STD, "LMDG_LM": L.LM, "LMDG_RLM": L.RLM, "LMDG_P0": L.P0, "LMDG_FP64": L.FP64,
              "LMDG_FP32": L.FP32, "LMDG_FP32_BF16STORE": L.FP32_BF16STORE, "LMDG_SWEEP_SOURCE": L.SWEEP_SOURCE,
              "LMDG_SWEEP_FP32": L.SWEEP_FP32, "LMDG_SWEEP_STORE": L.SWEEP_STORE, "LMDG_HOST_PTRS": L.HOST_PTRS,
              "LMDG_SWEEP_F32X2": L.SWEEP_F32X2, "LMDG_SOLVE_EXACT_REF": L.SOLVE_EXACT_REF,
              "LMDG_RESID_FP64": L.RESID_FP64, "LMDG_RESID_F32X2": L.RESID_F32X2,
              "LMDG_ERR_TIMEOUT": L.ERR_TIMEOUT, "LMDG_ERR_NOTCONV": L.ERR_NOTCONV, "LMDG_ERR_STATE": L.ERR_STATE}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "lmdg.h"', "int main(void) {"]
    for cname, py in structs.items():
        src.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            src.append(f'  printf("off {cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    for name in consts:
        src.append(f'  printf("const {name} %d\\n", (int){name});')
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        kind, *rest = line.split()
        if kind == "size":
            assert ctypes.sizeof(structs[rest[0]]) == int(rest[1]), line
        elif kind == "off":
            assert getattr(structs[rest[0]], rest[1]).offset == int(rest[2]), line
        else:
            assert consts[rest[0]] == int(rest[1]), line

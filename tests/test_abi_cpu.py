"""CPU-only checks of the boundary: the library builds, loads and exports
every function include/qsim.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\*?\s*\b(sim_[a-z0-9_]+|qsim_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1612_08091_gb300.build import build

    lib_path = build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "sim_apply" in names and "sim_expect" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_build_info_and_workspace_size():
    from paper_1612_08091_gb300 import load

    lib = load()
    assert b"sm_103a" in lib.qsim_build_info()
    sz = ctypes.c_size_t()
    assert lib.sim_workspace_bytes(20, 0, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.sim_workspace_bytes(0, 0, ctypes.byref(sz)) == 1  # EINVAL
    assert lib.sim_workspace_bytes(20, 7, ctypes.byref(sz)) == 1


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1612_08091_gb300 import Simulator

    with pytest.raises(RuntimeError):
        Simulator(4)


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1612_08091_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:import|from)\s+(\w+)", text, flags=re.M), f
                assert "qsim_oracle" not in text, f

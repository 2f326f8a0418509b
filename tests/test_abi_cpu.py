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


def declaration_comments():
    """Each function declared in include/*.h with the comment block that
    governs it: the nearest comment above the declaration, where consecutive
    declarations without a comment between them share the one above the
    first."""
    out = {}
    decl = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\*?\s*\b(sim_[a-z0-9_]+|qsim_[a-z0-9_]+)\s*\(")
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", h)).read().split("\n")
        for i, line in enumerate(lines):
            m = decl.match(line)
            if not m:
                continue
            j = i - 1
            # skip earlier declarations of the same group (and their continuation lines)
            while j >= 0 and "*/" not in lines[j] and lines[j].strip():
                j -= 1
            if j < 0 or "*/" not in lines[j]:
                out[m.group(1)] = ""
                continue
            k = j
            while k >= 0 and "/*" not in lines[k]:
                k -= 1
            text = " ".join(re.sub(r"^\s*(/\*+|\*+/?)?", "", l) for l in lines[k:j + 1])
            out[m.group(1)] = re.sub(r"\s+", " ", text)
    return out


def test_every_declaration_cites_its_passage():
    """Every entry point of the boundary names the passage of the paper that
    defines its operation (a section, figure or appendix), or says that the
    paper has no counterpart."""
    comments = declaration_comments()
    assert set(comments) == set(declared_functions())
    marker = re.compile(r"Sec\.\s*\d|Appendix\s+A|Fig\.\s*\d|not in the paper|The paper has no counterpart",
                        re.I)
    bad = sorted(name for name, c in comments.items() if not marker.search(c))
    assert not bad, bad
    # the calls that carry the paper's operations cite a passage, not only "not in the paper"
    for name in ("sim_create", "sim_destroy", "sim_apply", "sim_flush", "sim_prob", "sim_probs_all",
                 "sim_measure", "sim_collapse", "sim_measure_all", "sim_get_amplitudes", "sim_apply_permutation",
                 "sim_set_fusion"):
        assert re.search(r"Sec\.\s*\d|Appendix\s+A", comments[name]), name
    assert re.search(r"not in the paper", comments["sim_expect"], re.I)

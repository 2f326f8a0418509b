"""Host logic of the fusion planner, checked on the CPU: tests/planner_check.cpp
is compiled together with the library's planner.cpp (g++, no GPU) and run;
it compares fused block matrices with an independent element-wise embedding
of their gates and checks greedy plans of random circuits for coverage,
program order and block widths."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_planner_host_logic(tmp_path):
    gxx = shutil.which("g++")
    inc = cuda_include()
    if not gxx or not inc:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path / "planner_check")
    cmd = [gxx, "-O1", "-std=c++17", "-I", inc, os.path.join(ROOT, "tests", "planner_check.cpp"),
           os.path.join(ROOT, "paper_1612_08091_gb300", "csrc", "planner.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr

"""Compile the oracle's C core into a shared object next to its source.

Test infrastructure only (see the package docstring).  Plain gcc, OpenMP for
the loop over basis indices, no architecture-specific flags so that the same
source builds on x86_64 and aarch64 hosts.
"""
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()


def library_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Build ``liboracle.so`` if it is missing or older than its source."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + ".tmp.%d" % os.getpid()
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB

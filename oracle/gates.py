"""The oracle's gate matrices, each written from its textbook definition.

Test infrastructure only.  Convention (shared with the whole project, not
fixed by the paper): for a gate on targets ``(t0, t1, ...)`` the matrix row
index has bit j equal to qubit ``t_j``.

Gates named in the paper: H, X, Z, Rx (Sec. 4), CNOT and controlled X/Z
(Appendix A.1), R(phi) = diag(1, e^{i phi}) (Appendix A.3), multi-controlled Z
(Appendix A.2).  U3, RY, RZ, Y, S, T and SWAP are the standard definitions
used by the synthetic workloads.
"""
import math

import numpy as np

SQ2 = 1.0 / math.sqrt(2.0)


def H():
    return np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=np.complex128)


def X():
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def Y():
    return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def Z():
    return np.array([[1, 0], [0, -1]], dtype=np.complex128)


def S():
    return np.array([[1, 0], [0, 1j]], dtype=np.complex128)


def T():
    return np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128)


def RX(theta):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def RY(theta):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def RZ(phi):
    return np.array([[np.exp(-0.5j * phi), 0], [0, np.exp(0.5j * phi)]], dtype=np.complex128)


def R(phi):
    """Phase shift diag(1, e^{i phi}) (the R gate of the paper's Shor listing)."""
    return np.array([[1, 0], [0, np.exp(1j * phi)]], dtype=np.complex128)


def U3(theta, phi, lam):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array(
        [[c, -np.exp(1j * lam) * s], [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]],
        dtype=np.complex128,
    )


def SWAP():
    """Exchange of the two target qubits: |r=1> <-> |r=2> in the target index."""
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[3, 3] = 1
    m[1, 2] = m[2, 1] = 1
    return m


_NAMED = {"H": H, "X": X, "Y": Y, "Z": Z, "S": S, "T": T, "SWAP": SWAP}
_PARAM = {"RX": RX, "RY": RY, "RZ": RZ, "R": R, "U3": U3}


def matrix(kind, params=()):
    """Matrix of a gate given by its name and parameters; ``MAT`` carries an
    explicit matrix in ``params[0]``."""
    if kind == "MAT":
        return np.asarray(params[0], dtype=np.complex128)
    if kind in _NAMED:
        return _NAMED[kind]()
    if kind in _PARAM:
        return _PARAM[kind](*params)
    raise ValueError("unknown gate kind %r" % (kind,))

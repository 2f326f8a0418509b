"""Gate matrices for the GPU library's Python binding.

Convention: for a gate on targets (t0, t1, ...) bit j of the matrix row or
column index is the value of qubit t_j.  Matrices are complex128 numpy arrays,
row-major, handed to ``sim_apply`` as interleaved (re, im) doubles.

Gates from the ProjectQ paper: H, X, Z and Rx (Sec. 4), controlled X/Z
(Appendix A.1), the phase shift R(phi) (Appendix A.3) and the multi-controlled
Z of the Grover example (Appendix A.2).  U3, RY, RZ, Y, S, T and SWAP are the
standard definitions used by the synthetic workloads.
"""
import cmath
import math

import numpy as np

_INV_SQRT2 = math.sqrt(0.5)


def _m(rows):
    return np.array(rows, dtype=np.complex128)


def hadamard():
    return _m([[_INV_SQRT2, _INV_SQRT2], [_INV_SQRT2, -_INV_SQRT2]])


def pauli_x():
    return _m([[0, 1], [1, 0]])


def pauli_y():
    return _m([[0, -1j], [1j, 0]])


def pauli_z():
    return _m([[1, 0], [0, -1]])


def phase(phi):
    """R(phi) = diag(1, e^{i phi})."""
    return _m([[1, 0], [0, cmath.exp(1j * phi)]])


def rot_x(theta):
    h = 0.5 * theta
    return _m([[math.cos(h), -1j * math.sin(h)], [-1j * math.sin(h), math.cos(h)]])


def rot_y(theta):
    h = 0.5 * theta
    return _m([[math.cos(h), -math.sin(h)], [math.sin(h), math.cos(h)]])


def rot_z(phi):
    return _m([[cmath.exp(-0.5j * phi), 0], [0, cmath.exp(0.5j * phi)]])


def u3(theta, phi, lam):
    """U3 = RZ(phi) RY(theta) RZ(lam) up to the global phase e^{i(phi+lam)/2}."""
    c, s = math.cos(0.5 * theta), math.sin(0.5 * theta)
    return _m([[c, -cmath.exp(1j * lam) * s], [cmath.exp(1j * phi) * s, cmath.exp(1j * (phi + lam)) * c]])


def swap():
    out = np.eye(4, dtype=np.complex128)
    out[[1, 2]] = out[[2, 1]]
    return out


_FIXED = {
    "H": hadamard, "X": pauli_x, "Y": pauli_y, "Z": pauli_z, "SWAP": swap,
    "S": lambda: phase(math.pi / 2), "T": lambda: phase(math.pi / 4),
}
_PARAMETRIC = {"RX": rot_x, "RY": rot_y, "RZ": rot_z, "R": phase, "U3": u3}


def gate_matrix(kind, params=()):
    if kind == "MAT":
        return np.asarray(params[0], dtype=np.complex128)
    if kind in _FIXED:
        return _FIXED[kind]()
    if kind in _PARAMETRIC:
        return _PARAMETRIC[kind](*params)
    raise ValueError("unknown gate %r" % (kind,))

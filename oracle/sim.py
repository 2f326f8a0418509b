"""ctypes wrapper around the C oracle plus the slow Pauli-sum expectation.

Test infrastructure only.  Every method is a direct call of one C routine
(see ``qsim_oracle.c``) or, for expectation values, the definition
<psi| P |psi> with P applied factor by factor as ordinary gates.
"""
import ctypes

import numpy as np

from . import gates as G
from .build import build

_lib = None
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("oracle %s failed with code %d" % (what, code))
        self.code = code


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.or_apply.argtypes = [vp, ctypes.c_int, vp, _c_int_p, ctypes.c_int, _c_int_p, ctypes.c_int]
        lib.or_norm2.argtypes = [vp, ctypes.c_int]
        lib.or_norm2.restype = ctypes.c_double
        lib.or_prob_bits.argtypes = [vp, ctypes.c_int, _c_int_p, ctypes.c_int, _c_int_p, _c_dbl_p]
        lib.or_collapse.argtypes = [vp, ctypes.c_int, _c_int_p, ctypes.c_int, _c_int_p, _c_dbl_p]
        lib.or_measure.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _c_int_p, _c_dbl_p]
        lib.or_measure_all.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]
        lib.or_inner.argtypes = [vp, vp, ctypes.c_int, _c_dbl_p, _c_dbl_p]
        lib.or_inner.restype = None
        lib.or_set_basis.argtypes = [vp, ctypes.c_int, ctypes.c_uint64]
        _lib = lib
    return _lib


def _ints(seq):
    seq = [int(v) for v in seq]
    arr = (ctypes.c_int * max(1, len(seq)))(*seq)
    return arr, len(seq)


def _check(rc, what):
    if rc != 0:
        raise OracleError(rc, what)


class OracleSim:
    """An n-qubit register held as a contiguous complex128 numpy array."""

    def __init__(self, n, basis=0, psi=None):
        self.lib = _load()
        self.n = int(n)
        if psi is not None:
            self.psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
            assert self.psi.shape == (1 << self.n,)
        else:
            self.psi = np.zeros(1 << self.n, dtype=np.complex128)
            self.psi[int(basis)] = 1.0

    def _p(self, arr=None):
        a = self.psi if arr is None else arr
        return a.ctypes.data_as(ctypes.c_void_p)

    # -- gates -------------------------------------------------------------
    def apply(self, U, targets, controls=()):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        k = len(targets)
        if U.shape != (1 << k, 1 << k):
            raise ValueError("matrix shape %s does not match %d targets" % (U.shape, k))
        t, nt = _ints(targets)
        c, nc = _ints(controls)
        _check(self.lib.or_apply(self._p(), self.n, U.ctypes.data_as(ctypes.c_void_p), t, nt, c, nc), "apply")

    def apply_op(self, op):
        self.apply(G.matrix(op.kind, op.params), op.targets, op.controls)

    def apply_permutation(self, perm, qubits, controls=()):
        """Emulated classical bijection on a register (bit j of the register
        value is qubits[j]), from its definition: where all controls are 1,
        the amplitude of register value x moves to register value perm[x]."""
        perm = np.asarray(perm, dtype=np.int64)
        N = 1 << self.n
        idx = np.arange(N, dtype=np.int64)
        val = np.zeros(N, dtype=np.int64)
        regmask = 0
        for j, q in enumerate(qubits):
            val |= ((idx >> q) & 1) << j
            regmask |= 1 << q
        on = np.ones(N, dtype=bool)
        for c in controls:
            on &= ((idx >> c) & 1) == 1
        fv = perm[val]
        dest = idx & ~regmask
        for j, q in enumerate(qubits):
            dest |= ((fv >> j) & 1) << q
        out = self.psi.copy()
        out[dest[on]] = self.psi[on]
        self.psi = out

    # -- reads -------------------------------------------------------------
    def norm2(self):
        return float(self.lib.or_norm2(self._p(), self.n))

    def prob_bits(self, qubits, bits):
        q, m = _ints(qubits)
        b, _ = _ints(bits)
        out = ctypes.c_double()
        _check(self.lib.or_prob_bits(self._p(), self.n, q, m, b, ctypes.byref(out)), "prob_bits")
        return out.value

    def prob1(self, q):
        """P(qubit q = 1)."""
        return self.prob_bits([q], [1])

    def probs_all(self):
        return np.array([self.prob1(q) for q in range(self.n)])

    # -- measurement -------------------------------------------------------
    def collapse(self, qubits, bits):
        q, m = _ints(qubits)
        b, _ = _ints(bits)
        p = ctypes.c_double()
        _check(self.lib.or_collapse(self._p(), self.n, q, m, b, ctypes.byref(p)), "collapse")
        return p.value

    def measure(self, q, u):
        out = ctypes.c_int()
        p = ctypes.c_double()
        _check(self.lib.or_measure(self._p(), self.n, int(q), float(u), ctypes.byref(out), ctypes.byref(p)), "measure")
        return out.value

    def measure_all(self, u):
        out = ctypes.c_uint64()
        _check(self.lib.or_measure_all(self._p(), self.n, float(u), ctypes.byref(out)), "measure_all")
        return int(out.value)

    # -- observables -------------------------------------------------------
    def inner(self, other):
        """<self|other> for another complex128 array of the same length."""
        other = np.ascontiguousarray(other, dtype=np.complex128)
        re, im = ctypes.c_double(), ctypes.c_double()
        self.lib.or_inner(self._p(), self._p(other), self.n, ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    def expect(self, terms):
        """<psi| sum_k c_k P_k |psi> for terms (c_k, xmask_k, zmask_k).

        Qubit q of P_k is Y if bit q is set in both masks, X if only in
        xmask, Z if only in zmask, identity otherwise.  Each P_k is applied
        factor by factor to a copy of psi with the ordinary gate routine."""
        total = 0.0
        for coeff, xmask, zmask in terms:
            phi = OracleSim(self.n, psi=self.psi)
            for q in range(self.n):
                xb, zb = (int(xmask) >> q) & 1, (int(zmask) >> q) & 1
                if xb and zb:
                    phi.apply(G.Y(), [q])
                elif xb:
                    phi.apply(G.X(), [q])
                elif zb:
                    phi.apply(G.Z(), [q])
            total += float(coeff) * self.inner(phi.psi).real
        return total


def run_ops(sim, ops):
    """Apply a sequence of circuit ops (see ``circuitgen``) in program order."""
    for op in ops:
        sim.apply_op(op)
    return sim

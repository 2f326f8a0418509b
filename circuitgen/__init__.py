"""Seeded synthetic workloads: circuit descriptions, observables and draws.

This module is the one thing the FP64 oracle and the CUDA library both
consume.  It holds no arithmetic of the simulation method: it only draws
seeded random numbers and lists gates by name, qubits and parameters.  Each
side turns a gate name into a matrix with its own code.

An op is ``Op(kind, targets, controls, params)``:
  kind      gate name ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "R",
            "U3", "SWAP") or "MAT" with an explicit matrix in params[0];
  targets   tuple of target qubits (bit j of the matrix index is targets[j]);
  controls  tuple of control qubits (the gate acts where all are |1>);
  params    tuple of angles (or the matrix for "MAT").

A Pauli term is ``(coeff, xmask, zmask)``: qubit q carries Y when bit q is set
in both masks, X when only in xmask, Z when only in zmask.

Default seeds: 1612 (12-qubit random circuit), 8091 (30/32-qubit random and
QFT), 2016 (variational batch), 2017 (Grover), 2018 (held-out planner
circuits); uniform draws for measurements use seed + 1.
"""
import math
from collections import namedtuple

import numpy as np

Op = namedtuple("Op", ["kind", "targets", "controls", "params"])


def op(kind, targets, controls=(), params=()):
    return Op(kind, tuple(int(t) for t in targets), tuple(int(c) for c in controls), tuple(params))


# ---------------------------------------------------------------------------
# random U3 + CNOT brickwork
# ---------------------------------------------------------------------------
def random_u3_brickwork(n, depth, seed):
    """``depth`` layers; each layer is U3(theta, phi, lambda) on every qubit
    (angles uniform in [0, 2 pi), drawn per qubit in the order theta, phi,
    lambda) followed by CNOTs on pairs (0,1),(2,3),... in even layers and
    (1,2),(3,4),... in odd layers, control = lower qubit."""
    rng = np.random.default_rng(seed)
    ops = []
    for layer in range(depth):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            ops.append(op("U3", (q,), (), (float(ang[q, 0]), float(ang[q, 1]), float(ang[q, 2]))))
        for a in range(layer % 2, n - 1, 2):
            ops.append(op("X", (a + 1,), (a,)))
    return ops


def inverse_ops(ops):
    """The inverse circuit: reversed order, each gate replaced by its inverse.
    Only kinds whose inverse is again a named gate are supported."""
    inv = []
    for o in reversed(ops):
        k, p = o.kind, o.params
        if k in ("H", "X", "Y", "Z", "SWAP"):
            inv.append(o)
        elif k in ("RX", "RY", "RZ", "R"):
            inv.append(Op(k, o.targets, o.controls, (-p[0],)))
        elif k == "U3":
            theta, phi, lam = p
            inv.append(Op("U3", o.targets, o.controls, (-theta, -lam, -phi)))
        elif k == "S":
            inv.append(Op("R", o.targets, o.controls, (-math.pi / 2,)))
        elif k == "T":
            inv.append(Op("R", o.targets, o.controls, (-math.pi / 4,)))
        else:
            raise ValueError("no named inverse for %r" % (k,))
    return inv


# ---------------------------------------------------------------------------
# QFT
# ---------------------------------------------------------------------------
def qft_ops(n, swaps=True):
    """Quantum Fourier transform on qubits 0..n-1 (qubit n-1 most significant):
    for j = n-1 down to 0, H on j then R(pi / 2^(j-k)) on j controlled by k for
    k = j-1 down to 0; then SWAP(i, n-1-i).  Maps |x> to
    2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>."""
    ops = []
    for j in range(n - 1, -1, -1):
        ops.append(op("H", (j,)))
        for k in range(j - 1, -1, -1):
            ops.append(op("R", (j,), (k,), (math.pi / float(1 << (j - k)),)))
    if swaps:
        for i in range(n // 2):
            ops.append(op("SWAP", (i, n - 1 - i)))
    return ops


def basis_prep_ops(x, n):
    """X on every qubit whose bit in x is 1 (prepares |x> from |0...0>)."""
    return [op("X", (q,)) for q in range(n) if (int(x) >> q) & 1]


def ripple_adder_ops(m, reps=1):
    """A ripple-carry adder of two m-bit registers made of CNOT and Toffoli
    gates only (the MAJ / UMA construction): qubit 0 is the incoming carry
    (left at 0), a_i = qubit 2i+1, b_i = qubit 2i+2, and qubit 2m+1 receives
    the outgoing carry.  One application maps |a, b, z> to |a, (a + b) mod
    2^m, z ^ carry>; the sequence is repeated reps times."""
    A = lambda i: 2 * i + 1
    B = lambda i: 2 * i + 2
    ops = []

    def maj(c, b, a):
        ops.extend([op("X", (b,), (a,)), op("X", (c,), (a,)), op("X", (a,), (c, b))])

    def uma(c, b, a):
        ops.extend([op("X", (a,), (c, b)), op("X", (c,), (a,)), op("X", (b,), (c,))])

    for _ in range(reps):
        maj(0, B(0), A(0))
        for i in range(1, m):
            maj(A(i - 1), B(i), A(i))
        ops.append(op("X", (2 * m + 1,), (A(m - 1),)))
        for i in range(m - 1, 0, -1):
            uma(A(i - 1), B(i), A(i))
        uma(0, B(0), A(0))
    return ops


def adder_basis_index(m, a, b, z=0):
    """Register index of |a, b, z> in the layout of ripple_adder_ops."""
    x = 0
    for i in range(m):
        x |= ((a >> i) & 1) << (2 * i + 1)
        x |= ((b >> i) & 1) << (2 * i + 2)
    return x | (z << (2 * m + 1))


def random_basis_state(n, seed):
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, 1 << n, dtype=np.uint64))


# ---------------------------------------------------------------------------
# Grover search (phase oracle + reflection about the uniform superposition)
# ---------------------------------------------------------------------------
def grover_iterations(n):
    return int(math.floor(math.pi / 4.0 * math.sqrt(float(1 << n))))


def grover_marked(n, seed):
    return random_basis_state(n, seed)


def grover_iteration_ops(n, marked):
    """One iteration: oracle -1 on |marked> (X on the zero bits of marked,
    Z on qubit n-1 controlled by qubits 0..n-2, X again), then the
    reflection H^n X^n C^{n-1}Z X^n H^n."""
    flip = [op("X", (q,)) for q in range(n) if not (int(marked) >> q) & 1]
    mcz = op("Z", (n - 1,), tuple(range(n - 1)))
    ops = list(flip) + [mcz] + list(flip)
    ops += [op("H", (q,)) for q in range(n)] + [op("X", (q,)) for q in range(n)]
    ops += [mcz]
    ops += [op("X", (q,)) for q in range(n)] + [op("H", (q,)) for q in range(n)]
    return ops


def grover_ops(n, marked, iterations=None):
    r = grover_iterations(n) if iterations is None else int(iterations)
    ops = [op("H", (q,)) for q in range(n)]
    body = grover_iteration_ops(n, marked)
    for _ in range(r):
        ops += body
    return ops


# ---------------------------------------------------------------------------
# hardware-efficient ansatz batch and the transverse-field Ising energy
# ---------------------------------------------------------------------------
def hea_ops(n, ry, rz):
    """Layers l: RY(ry[l][q]) on all q, RZ(rz[l][q]) on all q, then
    CNOT(q -> q+1) for q = 0..n-2 in order.  Starts from |0...0>."""
    ops = []
    for l in range(len(ry)):
        ops += [op("RY", (q,), (), (float(ry[l][q]),)) for q in range(n)]
        ops += [op("RZ", (q,), (), (float(rz[l][q]),)) for q in range(n)]
        ops += [op("X", (q + 1,), (q,)) for q in range(n - 1)]
    return ops


def hea_batch(count, seed, nmin=10, nmax=20, lmin=2, lmax=8):
    """``count`` circuits: n uniform in [nmin, nmax], L uniform in [lmin,
    lmax], angles uniform in [-pi, pi] drawn RY-then-RZ per layer.
    Returns a list of dicts with keys n, L, ry (L x n), rz (L x n)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        L = int(rng.integers(lmin, lmax + 1))
        ry = np.empty((L, n))
        rz = np.empty((L, n))
        for l in range(L):
            ry[l] = rng.uniform(-math.pi, math.pi, size=n)
            rz[l] = rng.uniform(-math.pi, math.pi, size=n)
        out.append({"n": n, "L": L, "ry": ry, "rz": rz})
    return out


def zz_chain_terms(n, coeff=1.0):
    """sum_{i=0}^{n-2} Z_i Z_{i+1} (open chain)."""
    return [(coeff, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]


def tfim_terms(n, h=0.7):
    """-sum_i Z_i Z_{i+1} - h sum_i X_i (open chain)."""
    return zz_chain_terms(n, -1.0) + [(-h, 1 << i, 0) for i in range(n)]


# ---------------------------------------------------------------------------
# the simulator-comparison circuit of the paper (Sec. 4.3.2): H transform,
# chain of controlled z-rotations, H transform
# ---------------------------------------------------------------------------
def hadamard_crz_chain(n, seed):
    rng = np.random.default_rng(seed)
    phis = rng.uniform(0.0, 2.0 * math.pi, size=max(0, n - 1))
    ops = [op("H", (q,)) for q in range(n)]
    ops += [op("RZ", (i + 1,), (i,), (float(phis[i]),)) for i in range(n - 1)]
    ops += [op("H", (q,)) for q in range(n)]
    return ops


# ---------------------------------------------------------------------------
# draws and misc inputs
# ---------------------------------------------------------------------------
def uniform_draws(seed, count):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=count)


def random_unitary(dim, seed):
    """Haar-ish random unitary from the QR factorisation of a complex Gaussian
    matrix (an input matrix, not part of the method)."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def workload_random12(seed=1612):
    """The 12-qubit check: 20 layers of the random brickwork, then P(q=1) for
    all q, <sum Z_i Z_{i+1}> and a full-register sample with a fixed draw."""
    n, depth = 12, 20
    return {
        "n": n,
        "ops": random_u3_brickwork(n, depth, seed),
        "terms": zz_chain_terms(n),
        "u": float(uniform_draws(seed + 1, 1)[0]),
    }

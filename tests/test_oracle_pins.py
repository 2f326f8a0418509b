"""Pins of the FP64 oracle against things other than itself (CPU only).

Each pin is chosen so that a plausible slip in the oracle fails it: a
transposed matrix or wrong target order (brute-force Kronecker and
element-by-element operator definitions), a dropped control (textbook CNOT,
teleportation), a wrong phase sign (QFT closed form, GHZ <YYX>), a wrong
normalisation (Grover closed form, collapse), a wrong cumulative-sum rule
(measure-all against numpy's cumsum/searchsorted).
"""
import math
import os

import numpy as np
import pytest

import circuitgen as cg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sim(oracle_mod, n, psi=None, basis=0):
    return oracle_mod.OracleSim(n, basis=basis, psi=psi)


# ---------------------------------------------------------------------------
# gate application against operators built independently
# ---------------------------------------------------------------------------
def kron_embed(U, q, n):
    """Textbook embedding of a one-qubit operator: I (x) ... (x) U (x) ... (x) I,
    qubit 0 the rightmost (least significant) factor."""
    left = np.eye(1 << (n - 1 - q))
    right = np.eye(1 << q)
    return np.kron(left, np.kron(U, right))


def full_operator(U, targets, controls, n):
    """<i|G|j> straight from the definition: identity on qubits outside the
    targets, U on the target bits where every control bit of j is 1."""
    N = 1 << n
    tmask = sum(1 << t for t in targets)
    cmask = sum(1 << c for c in controls)

    def r_of(i):
        return sum(((i >> t) & 1) << j for j, t in enumerate(targets))

    M = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            if (i & ~tmask) != (j & ~tmask):
                continue
            if (j & cmask) == cmask:
                M[i, j] = U[r_of(i), r_of(j)]
            else:
                M[i, j] = 1.0 if i == j else 0.0
    return M


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_single_qubit_matches_kronecker(oracle_mod, n):
    for q in range(n):
        U = cg.random_unitary(2, seed=100 * n + q)
        psi = cg.random_state(n, seed=7 + q)
        s = _sim(oracle_mod, n, psi=psi)
        s.apply(U, [q])
        np.testing.assert_allclose(s.psi, kron_embed(U, q, n) @ psi, atol=1e-13)


@pytest.mark.parametrize(
    "n,targets,controls",
    [
        (2, (0,), (1,)),
        (3, (2, 0), ()),
        (3, (0, 2), ()),
        (4, (1, 3), (0,)),
        (5, (4, 1, 2), ()),
        (5, (0,), (2, 4)),
        (6, (3, 5, 0), (1, 4)),
        (6, (5, 4), (3, 2, 1)),
        (6, (2, 1, 5, 0), ()),
    ],
)
def test_dense_controlled_matches_definition(oracle_mod, n, targets, controls):
    U = cg.random_unitary(1 << len(targets), seed=len(targets) * 31 + n)
    psi = cg.random_state(n, seed=n + 11)
    s = _sim(oracle_mod, n, psi=psi)
    s.apply(U, targets, controls)
    np.testing.assert_allclose(s.psi, full_operator(U, targets, controls, n) @ psi, atol=1e-13)


def test_textbook_cnot_and_swap(oracle_mod):
    # basis index = 2*q1 + q0.  CNOT with control q0, target q1 maps
    # |q1 q0> = |0 1> (index 1) to |1 1> (index 3) and back.
    cnot = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=np.complex128)
    swap = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
    psi = cg.random_state(2, seed=3)
    s = _sim(oracle_mod, 2, psi=psi)
    s.apply_op(cg.op("X", (1,), (0,)))
    np.testing.assert_allclose(s.psi, cnot @ psi, atol=1e-14)
    s = _sim(oracle_mod, 2, psi=psi)
    s.apply_op(cg.op("SWAP", (0, 1)))
    np.testing.assert_allclose(s.psi, swap @ psi, atol=1e-14)


def test_gate_library_identities(oracle_mod):
    G = oracle_mod.gates
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    np.testing.assert_allclose(G.U3(math.pi / 2, 0, math.pi), h, atol=1e-15)
    np.testing.assert_allclose(G.U3(math.pi, 0, math.pi), [[0, 1], [1, 0]], atol=1e-15)
    for th in (0.3, 1.7, -2.2):
        np.testing.assert_allclose(G.U3(th, 0, 0), G.RY(th), atol=1e-15)
        np.testing.assert_allclose(G.U3(th, -math.pi / 2, math.pi / 2), G.RX(th), atol=1e-15)
        # RZ equals the phase gate R up to the global phase e^{-i th/2}
        np.testing.assert_allclose(G.RZ(th), np.exp(-0.5j * th) * G.R(th), atol=1e-15)
    np.testing.assert_allclose(G.R(math.pi / 2), G.S(), atol=1e-15)
    np.testing.assert_allclose(G.R(math.pi / 4), G.T(), atol=1e-15)
    np.testing.assert_allclose(G.Y(), 1j * G.X() @ G.Z(), atol=1e-15)
    for U in (G.U3(0.4, 1.1, -0.7), G.RX(0.2), G.RY(1.3), G.RZ(0.9), G.SWAP()):
        np.testing.assert_allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 4, 9])
def test_hadamard_transform_uniform(oracle_mod, n):
    s = _sim(oracle_mod, n)
    cg_ops = [cg.op("H", (q,)) for q in range(n)]
    oracle_mod.run_ops(s, cg_ops)
    np.testing.assert_allclose(s.psi, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-14)


def test_ghz_matches_paper_histogram(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "entangle3_histogram.txt")) if l[0] != "#"]
    want = {int(b, 2): float(p) for b, p in rows}
    s = _sim(oracle_mod, 3)
    oracle_mod.run_ops(s, [cg.op("H", (0,)), cg.op("X", (1,), (0,)), cg.op("X", (2,), (0,))])
    for idx, p in want.items():
        assert abs(abs(s.psi[idx]) ** 2 - p) < 1e-15


@pytest.mark.parametrize("n,seed", [(3, 1), (6, 2), (10, 3), (13, 4)])
def test_qft_basis_state_closed_form(oracle_mod, n, seed):
    x = cg.random_basis_state(n, seed)
    N = 1 << n
    s = _sim(oracle_mod, n, basis=x)
    oracle_mod.run_ops(s, cg.qft_ops(n))
    y = np.arange(N, dtype=np.uint64)
    r = (np.uint64(x) * y) % np.uint64(N)  # exact integer phase numerator
    want = np.exp(2j * np.pi * r.astype(np.float64) / N) / math.sqrt(N)
    np.testing.assert_allclose(s.psi, want, atol=1e-12)


@pytest.mark.parametrize("n,depth", [(6, 5), (10, 8)])
def test_circuit_then_inverse_returns_zero_state(oracle_mod, n, depth):
    ops = cg.random_u3_brickwork(n, depth, seed=17)
    s = _sim(oracle_mod, n)
    oracle_mod.run_ops(s, ops)
    assert abs(s.norm2() - 1.0) < 1e-12
    assert abs(s.psi[0]) < 0.99  # the forward circuit really moved the state
    oracle_mod.run_ops(s, cg.inverse_ops(ops))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = 1
    np.testing.assert_allclose(s.psi, want, atol=1e-12)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_grover_closed_form(oracle_mod, n):
    marked = cg.grover_marked(n, seed=2017 + n)
    r = cg.grover_iterations(n)
    N = 1 << n
    s = _sim(oracle_mod, n)
    oracle_mod.run_ops(s, cg.grover_ops(n, marked))
    theta = math.asin(1.0 / math.sqrt(N))
    # the reflection used here is -(2|s><s| - I), so each iteration adds a
    # factor -1 to the textbook Grover state
    sign = (-1.0) ** r
    want = np.full(N, sign * math.cos((2 * r + 1) * theta) / math.sqrt(N - 1), dtype=np.complex128)
    want[marked] = sign * math.sin((2 * r + 1) * theta)
    np.testing.assert_allclose(s.psi, want, atol=1e-12)


# ---------------------------------------------------------------------------
# measurement
# ---------------------------------------------------------------------------
def test_rng_example(oracle_mod):
    rows = dict(l.split() for l in open(os.path.join(GOLDEN, "rng_h_measure.txt")) if l[0] != "#")
    p1 = float(rows["p1"])
    for u, want in [(0.0, 0), (0.49, 0), (0.51, 1), (0.999, 1)]:
        s = _sim(oracle_mod, 1)
        s.apply_op(cg.op("H", (0,)))
        assert abs(s.prob1(0) - p1) < 1e-15
        assert s.measure(0, u) == want
        assert abs(abs(s.psi[want]) - 1.0) < 1e-15 and abs(s.psi[1 - want]) == 0


def test_prob_and_collapse_match_numpy(oracle_mod):
    n = 7
    psi = cg.random_state(n, seed=5)
    idx = np.arange(1 << n)
    for qubits, bits in [((0,), (1,)), ((6,), (0,)), ((2, 5), (1, 0)), ((1, 3, 4), (1, 1, 0))]:
        sel = np.ones(1 << n, dtype=bool)
        for q, b in zip(qubits, bits):
            sel &= ((idx >> q) & 1) == b
        p = float(np.sum(np.abs(psi[sel]) ** 2))
        s = _sim(oracle_mod, n, psi=psi)
        assert abs(s.prob_bits(qubits, bits) - p) < 1e-14
        got_p = s.collapse(qubits, bits)
        assert abs(got_p - p) < 1e-14
        want = np.where(sel, psi / math.sqrt(p), 0)
        np.testing.assert_allclose(s.psi, want, atol=1e-14)


def test_zero_probability_collapse_is_rejected(oracle_mod):
    s = _sim(oracle_mod, 3, basis=0)
    before = s.psi.copy()
    with pytest.raises(oracle_mod.sim.OracleError):
        s.collapse([1], [1])
    np.testing.assert_array_equal(s.psi, before)


@pytest.mark.parametrize("outcome", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_teleportation(oracle_mod, outcome):
    # Appendix A.1: b1=qubit 0, b2=qubit 1, psi=qubit 2.
    U = cg.random_unitary(2, seed=99)
    s = _sim(oracle_mod, 3)
    s.apply(U, [2])  # Alice's state  U|0>
    ops = [
        cg.op("H", (0,)), cg.op("X", (1,), (0,)),  # Bell pair b1,b2
        cg.op("X", (0,), (2,)),  # CNOT psi -> b1
        cg.op("H", (2,)),
    ]
    oracle_mod.run_ops(s, ops)
    m_psi, m_b1 = outcome
    p = s.collapse([2, 0], [m_psi, m_b1])
    assert abs(p - 0.25) < 1e-14
    if m_b1:
        s.apply_op(cg.op("X", (1,)))
    if m_psi:
        s.apply_op(cg.op("Z", (1,)))
    # Bob's qubit (1) must now hold U|0>, the others are fixed at the outcome
    base = (m_psi << 2) | m_b1
    bob = np.array([s.psi[base], s.psi[base | 2]])
    np.testing.assert_allclose(bob, U[:, 0], atol=1e-14)


def test_measure_all_matches_numpy_search(oracle_mod):
    n = 8
    psi = cg.random_state(n, seed=12)
    w = np.abs(psi) ** 2
    cdf = np.cumsum(w)
    for u in cg.uniform_draws(77, 25):
        j = int(np.searchsorted(cdf, u * cdf[-1], side="right"))
        s = _sim(oracle_mod, n, psi=psi)
        got = s.measure_all(u)
        assert got == j
        assert abs(abs(s.psi[j]) - 1.0) < 1e-14
        assert abs(np.angle(s.psi[j]) - np.angle(psi[j])) < 1e-12
        assert np.count_nonzero(s.psi) == 1


def test_measure_all_basis_state(oracle_mod):
    for x in (0, 5, 127):
        for u in (0.0, 0.5, 0.999999):
            s = _sim(oracle_mod, 7, basis=x)
            assert s.measure_all(u) == x


def test_born_frequencies(oracle_mod):
    n = 3
    psi = cg.random_state(n, seed=8)
    w = np.abs(psi) ** 2
    draws = cg.uniform_draws(9, 4000)
    counts = np.zeros(1 << n)
    for u in draws:
        counts[_sim(oracle_mod, n, psi=psi).measure_all(u)] += 1
    expected = w * len(draws)
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    assert chi2 < 30.0  # 7 degrees of freedom; p < 1e-4 above this


# ---------------------------------------------------------------------------
# expectation values
# ---------------------------------------------------------------------------
PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def pauli_matrix(xmask, zmask, n):
    m = np.eye(1, dtype=np.complex128)
    for q in range(n - 1, -1, -1):  # qubit n-1 leftmost factor
        xb, zb = (xmask >> q) & 1, (zmask >> q) & 1
        m = np.kron(m, PAULI["Y" if xb and zb else "X" if xb else "Z" if zb else "I"])
    return m


def test_expect_matches_pauli_kronecker(oracle_mod):
    n = 5
    rng = np.random.default_rng(4)
    psi = cg.random_state(n, seed=21)
    terms = [(float(rng.normal()), int(rng.integers(0, 32)), int(rng.integers(0, 32))) for _ in range(12)]
    want = sum(c * np.vdot(psi, pauli_matrix(x, z, n) @ psi).real for c, x, z in terms)
    got = _sim(oracle_mod, n, psi=psi).expect(terms)
    assert abs(got - want) < 1e-13


def test_expect_closed_forms(oracle_mod):
    n = 6
    zero = _sim(oracle_mod, n)
    assert abs(zero.expect(cg.zz_chain_terms(n)) - (n - 1)) < 1e-14
    plus = _sim(oracle_mod, n)
    oracle_mod.run_ops(plus, [cg.op("H", (q,)) for q in range(n)])
    assert abs(plus.expect([(1.0, 1 << q, 0) for q in range(n)]) - n) < 1e-13
    assert abs(plus.expect(cg.tfim_terms(n)) - (-0.7 * n)) < 1e-13
    ghz = _sim(oracle_mod, n)
    oracle_mod.run_ops(ghz, [cg.op("H", (0,))] + [cg.op("X", (q,), (0,)) for q in range(1, n)])
    assert abs(ghz.expect(cg.zz_chain_terms(n)) - (n - 1)) < 1e-14
    assert abs(ghz.expect([(1.0, 1 << 2, 0)])) < 1e-14
    full = (1 << n) - 1
    assert abs(ghz.expect([(1.0, full, 0)]) - 1.0) < 1e-14
    # Y on qubits 0 and 1, X elsewhere: i*i = -1 on |1...1> <-> |0...0>
    assert abs(ghz.expect([(1.0, full, 0b11)]) + 1.0) < 1e-14


def test_semiclassical_phase_estimation_oracle(oracle_mod):
    """Appendix A.3's measure-and-reset loop (semi-classical inverse QFT) on
    the oracle: the phase k / 2^m of R(2 pi k / 2^m) on |1> comes out bit
    for bit, least significant first."""
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "semiclassical", os.path.join(os.path.dirname(__file__), "test_gpu_semiclassical.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    for m, k in [(3, 5), (5, 19), (7, 100)]:
        s = _sim(oracle_mod, 3)
        bits = mod.phase_estimation(s, m, k, cg.uniform_draws(k, m))
        assert bits == [(k >> j) & 1 for j in range(m)]


def test_permutation_emulation_pins(oracle_mod):
    """The oracle's register permutation (Sec. 4.3.3 emulation): identity,
    an inverse pair, and agreement with the permutation matrix applied as an
    ordinary (controlled) gate."""
    n = 6
    rng = np.random.default_rng(3)
    psi = cg.random_state(n, seed=33)
    s = _sim(oracle_mod, n, psi=psi)
    s.apply_permutation(np.arange(8), [4, 1, 2])
    np.testing.assert_array_equal(s.psi, psi)
    add5 = (np.arange(16) + 5) % 16
    sub5 = (np.arange(16) - 5) % 16
    s.apply_permutation(add5, [0, 2, 3, 5])
    assert np.max(np.abs(s.psi - psi)) > 0.1
    s.apply_permutation(sub5, [0, 2, 3, 5])
    np.testing.assert_allclose(s.psi, psi, atol=0)
    for qubits, controls in [((1, 3), ()), ((5, 0, 2), (4,)), ((2, 3, 4, 0), (1,))]:
        m = len(qubits)
        perm = rng.permutation(1 << m)
        P = np.zeros((1 << m, 1 << m))
        P[perm, np.arange(1 << m)] = 1.0  # column x has its 1 in row perm[x]
        a = _sim(oracle_mod, n, psi=psi)
        a.apply_permutation(perm, qubits, controls)
        b = _sim(oracle_mod, n, psi=psi)
        b.apply(P, qubits, controls)
        np.testing.assert_allclose(a.psi, b.psi, atol=1e-15)


@pytest.mark.parametrize("m", [3, 5])
def test_ripple_adder_adds(oracle_mod, m):
    """The CNOT / Toffoli ripple-carry adder on basis states: |a, b, 0> goes
    to |a, (a + b) mod 2^m, carry> with amplitude 1 (classical arithmetic
    fixes the result, independent of the oracle's gate code)."""
    n = 2 * m + 2
    rng = np.random.default_rng(m)
    for _ in range(6):
        a, b = (int(v) for v in rng.integers(0, 1 << m, 2))
        s = _sim(oracle_mod, n)
        s.psi[:] = 0
        s.psi[cg.adder_basis_index(m, a, b)] = 1.0
        oracle_mod.run_ops(s, cg.ripple_adder_ops(m))
        want = cg.adder_basis_index(m, a, (a + b) % (1 << m), (a + b) >> m)
        assert abs(s.psi[want] - 1.0) < 1e-15
        assert np.sum(np.abs(s.psi) ** 2) - abs(s.psi[want]) ** 2 < 1e-15

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances are stated in tests/helpers.py."""
import math

import numpy as np
import pytest

import circuitgen as cg
from helpers import TOL128_AMP, TOL64_INFID, TOL64_PROB, expect_tol, infidelity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1612_08091_gb300 as q

    q.load()
    return q


def make(qs, n, prec, fusion="none", kmax=5):
    return qs.Simulator(n, precision=prec, fusion=fusion, kmax=kmax)


def oracle_run(oracle_mod, n, ops, psi=None):
    s = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(s, ops)
    return s


def check_state(got, want, prec):
    if prec == "c128":
        assert np.max(np.abs(got - want)) <= TOL128_AMP
    else:
        assert infidelity(want, got) <= TOL64_INFID
        assert np.max(np.abs(got - want)) <= 1e-5


# ---------------------------------------------------------------------------
# single gates: every kind, placements across vector/tile boundaries
# ---------------------------------------------------------------------------
GATE_CASES = [
    ("H", (0,), ()), ("H", (1,), ()), ("H", (5,), ()), ("U3", (0,), ()), ("U3", (13,), ()),
    ("X", (1,), (0,)), ("X", (0,), (13,)), ("X", (7,), (2, 11)), ("Z", (13,), tuple(range(13))),
    ("R", (3,), (12,)), ("R", (0,), ()), ("RZ", (9,), ()), ("RZ", (4,), (0, 1)), ("Y", (6,), ()),
    ("SWAP", (0, 13), ()), ("SWAP", (2, 3), (7,)), ("MAT2", (5, 1), ()), ("MAT3", (0, 12, 6), (3,)),
    ("MAT4", (13, 2, 8, 0), ()), ("MAT5", (1, 3, 5, 7, 9), (11,)), ("MAT5", (13, 12, 11, 10, 0), ()),
]


def case_op(kind, targets, controls, seed):
    rng = np.random.default_rng(seed)
    if kind.startswith("MAT"):
        return cg.op("MAT", targets, controls, (cg.random_unitary(1 << len(targets), seed),))
    if kind == "U3":
        return cg.op("U3", targets, controls, tuple(rng.uniform(0, 2 * math.pi, 3)))
    if kind in ("R", "RZ"):
        return cg.op(kind, targets, controls, (float(rng.uniform(0, 2 * math.pi)),))
    return cg.op(kind, targets, controls)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("case", range(len(GATE_CASES)))
def test_single_gate(qs, oracle_mod, prec, case):
    n = 14
    kind, t, c = GATE_CASES[case]
    op = case_op(kind, t, c, seed=case)
    psi = cg.random_state(n, seed=100 + case)
    want = oracle_run(oracle_mod, n, [op], psi=psi).psi
    with make(qs, n, prec) as sim:
        sim.set_amplitudes(psi)
        sim.apply_op(op)
        got = sim.get_amplitudes()
    check_state(got, want, prec)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_exhaustive_small_placements(qs, oracle_mod, prec):
    n = 6
    rng = np.random.default_rng(5)
    psi = cg.random_state(n, seed=6)
    ops = []
    for t in range(n):
        for c in range(n):
            if c != t:
                ops.append(cg.op("U3", (t,), (c,), tuple(rng.uniform(0, 6.28, 3))))
        for t2 in range(n):
            if t2 != t:
                ops.append(cg.op("MAT", (t, t2), (), (cg.random_unitary(4, t * 7 + t2),)))
    want = oracle_run(oracle_mod, n, ops, psi=psi).psi
    with make(qs, n, prec) as sim:
        sim.set_amplitudes(psi)
        sim.run(ops)
        got = sim.get_amplitudes()
    if prec == "c128":
        assert np.max(np.abs(got - want)) <= TOL128_AMP
    else:
        assert infidelity(want, got) <= TOL64_INFID


# ---------------------------------------------------------------------------
# the 12-qubit random circuit with probabilities, <sum ZZ> and measure-all
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,fusion", [("c128", "none"), ("c64", "none"), ("c64", "greedy"), ("c128", "greedy")])
def test_random12_full_check(qs, oracle_mod, prec, fusion):
    w = cg.workload_random12()
    n = w["n"]
    ref = oracle_run(oracle_mod, n, w["ops"])
    with make(qs, n, prec, fusion) as sim:
        sim.run(w["ops"])
        got = sim.get_amplitudes()
        p1, nrm = sim.probs_all()
        e = sim.expect(w["terms"])
        check_state(got, ref.psi, prec)
        tol = 1e-11 if prec == "c128" else TOL64_PROB
        np.testing.assert_allclose(p1, ref.probs_all(), atol=tol)
        assert abs(nrm - 1.0) <= tol
        assert abs(e - ref.expect(w["terms"])) <= expect_tol(w["terms"], tol)
        j = sim.measure_all(w["u"])
    c = np.cumsum(np.abs(ref.psi) ** 2)
    jr = ref.measure_all(w["u"])
    # equal, or both sides of a cumulative-sum boundary within the rounding
    # of the amplitudes (complex128: FP64 sums of 2^12 terms)
    assert j == jr or abs(c[min(j, jr)] - w["u"] * c[-1]) < (1e-12 if prec == "c128" else 1e-6)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [3, 9, 10, 11, 16])
def test_probs_all_and_prob(qs, oracle_mod, prec, n):
    psi = cg.random_state(n, seed=n)
    ref = oracle_mod.OracleSim(n, psi=psi)
    with make(qs, n, prec) as sim:
        sim.set_amplitudes(psi)
        p1, nrm = sim.probs_all()
        tol = 1e-12 if prec == "c128" else 1e-6
        np.testing.assert_allclose(p1, ref.probs_all(), atol=tol)
        assert abs(nrm - ref.norm2()) <= tol
        for q in (0, n // 2, n - 1):
            assert abs(sim.prob(q) - ref.prob1(q)) <= tol


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [4, 12])
def test_expect_random_paulis(qs, oracle_mod, prec, n):
    rng = np.random.default_rng(n)
    psi = cg.random_state(n, seed=30 + n)
    terms = [(float(rng.normal()), int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))) for _ in range(20)]
    terms += [(0.5, 0, int(rng.integers(0, 1 << n))) for _ in range(5)] + cg.tfim_terms(n)
    ref = oracle_mod.OracleSim(n, psi=psi).expect(terms)
    with make(qs, n, prec) as sim:
        sim.set_amplitudes(psi)
        got = sim.expect(terms)
    tol = 1e-11 if prec == "c128" else TOL64_PROB
    assert abs(got - ref) <= expect_tol(terms, tol)


# ---------------------------------------------------------------------------
# measurement and collapse
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_measure_and_collapse(qs, oracle_mod, prec):
    n = 11
    psi = cg.random_state(n, seed=77)
    for q, u in [(0, 0.3), (5, 0.9), (10, 0.01)]:
        ref = oracle_mod.OracleSim(n, psi=psi)
        ref_before = oracle_mod.OracleSim(n, psi=psi)
        b_ref = ref.measure(q, u)
        p_ref = ref_before.prob1(q) if b_ref else 1.0 - ref_before.prob1(q)
        with make(qs, n, prec) as sim:
            sim.set_amplitudes(psi)
            b, p = sim.measure(q, u)
            got = sim.get_amplitudes()
        assert b == b_ref
        # the reported probability is the one that decided the outcome
        assert abs(p - p_ref) <= (1e-12 if prec == "c128" else 1e-6)
        check_state(got, ref.psi, prec)
    ref = oracle_mod.OracleSim(n, psi=psi)
    p_ref = ref.collapse([1, 4, 9], [1, 0, 1])
    with make(qs, n, prec) as sim:
        sim.set_amplitudes(psi)
        p = sim.collapse([1, 4, 9], [1, 0, 1])
        got = sim.get_amplitudes()
    assert abs(p - p_ref) <= (1e-12 if prec == "c128" else 1e-6)
    check_state(got, ref.psi, prec)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_measure_all_draws(qs, oracle_mod, prec):
    n = 13
    psi = cg.random_state(n, seed=4)
    for u in cg.uniform_draws(11, 6):
        ref = oracle_mod.OracleSim(n, psi=psi)
        jr = ref.measure_all(u)
        with make(qs, n, prec) as sim:
            sim.set_amplitudes(psi)
            j = sim.measure_all(u)
            got = sim.get_amplitudes()
        if j != jr:
            # only acceptable at a cumulative-sum boundary (rounding order;
            # complex128: FP64 sums of 2^13 terms, complex64: the amplitudes
            # themselves are rounded to FP32)
            w = np.abs(psi) ** 2
            c = np.cumsum(w)
            assert abs(c[min(j, jr)] - u * c[-1]) < (1e-12 if prec == "c128" else 1e-6)
        assert abs(abs(got[j]) - 1.0) < 1e-6 and np.count_nonzero(got) == 1


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_teleportation_and_rng(qs, prec):
    U = cg.random_unitary(2, seed=99)
    for m_psi in (0, 1):
        for m_b1 in (0, 1):
            with make(qs, 3, prec) as sim:
                sim.apply(U, [2])
                sim.run([cg.op("H", (0,)), cg.op("X", (1,), (0,)), cg.op("X", (0,), (2,)), cg.op("H", (2,))])
                p = sim.collapse([2, 0], [m_psi, m_b1])
                assert abs(p - 0.25) < 1e-6
                if m_b1:
                    sim.apply_op(cg.op("X", (1,)))
                if m_psi:
                    sim.apply_op(cg.op("Z", (1,)))
                a = sim.get_amplitudes()
            base = (m_psi << 2) | m_b1
            np.testing.assert_allclose([a[base], a[base | 2]], U[:, 0], atol=1e-6)
    with make(qs, 1, prec) as sim:
        sim.apply_op(cg.op("H", (0,)))
        assert abs(sim.prob(0) - 0.5) < 1e-7
        assert sim.measure(0, 0.4)[0] == 0


# ---------------------------------------------------------------------------
# closed forms and larger registers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,fusion", [("c128", "none"), ("c64", "greedy")])
def test_qft_closed_form(qs, prec, fusion):
    n = 18
    x = cg.random_basis_state(n, seed=3)
    with make(qs, n, prec, fusion) as sim:
        sim.run(cg.basis_prep_ops(x, n) + cg.qft_ops(n))
        got = sim.get_amplitudes()
    N = 1 << n
    y = np.arange(N, dtype=np.uint64)
    r = (np.uint64(x) * y) % np.uint64(N)
    want = np.exp(2j * np.pi * r.astype(np.float64) / N) / math.sqrt(N)
    check_state(got, want, prec)


@pytest.mark.parametrize("prec,fusion", [("c128", "none"), ("c64", "none"), ("c64", "greedy")])
def test_grover_closed_form(qs, prec, fusion):
    n = 10
    marked = cg.grover_marked(n, seed=2017)
    r = cg.grover_iterations(n)
    with make(qs, n, prec, fusion) as sim:
        sim.run(cg.grover_ops(n, marked))
        got = sim.get_amplitudes()
    theta = math.asin(2.0 ** (-n / 2))
    want = np.full(1 << n, math.cos((2 * r + 1) * theta) / math.sqrt((1 << n) - 1), dtype=np.complex128)
    want[marked] = math.sin((2 * r + 1) * theta)
    want *= (-1) ** r
    check_state(got, want, prec)


@pytest.mark.parametrize("prec,fusion,kmax", [("c128", "none", 5), ("c64", "greedy", 6), ("c64", "greedy", 5),
                                              ("c64", "greedy", 4), ("c64", "greedy", 2)])
def test_random_circuit_n20(qs, oracle_mod, prec, fusion, kmax):
    n = 20
    ops = cg.random_u3_brickwork(n, 10, seed=8091)
    ref = oracle_run(oracle_mod, n, ops)
    with make(qs, n, prec, fusion, kmax) as sim:
        sim.run(ops)
        got = sim.get_amplitudes()
        st = sim.stats()
    check_state(got, ref.psi, prec)
    if fusion == "greedy":
        assert st["passes"] < len(ops)


def test_errors_leave_state_unchanged(qs):
    n = 5
    psi = cg.random_state(n, seed=1)
    with make(qs, n, "c128") as sim:
        sim.set_amplitudes(psi)
        for args, status in [
            ((np.eye(2), [5]), "ERANGE"),
            ((np.eye(2), [1], [1]), "EDUP"),
            ((np.full((2, 2), np.nan), [1]), "ENONFINITE"),
            ((np.eye(64), [0, 1, 2, 3, 4, 5]), "EINVAL"),
        ]:
            with pytest.raises(qs.QsimError) as e:
                sim.apply(*args)
            assert e.value.status == status
        with pytest.raises(qs.QsimError) as e:
            sim.measure(0, 1.5)
        assert e.value.status == "EINVAL"
        np.testing.assert_allclose(sim.get_amplitudes(), psi, atol=0)
    with make(qs, 3, "c64") as sim:
        with pytest.raises(qs.QsimError) as e:
            sim.collapse([0], [1])
        assert e.value.status == "EZEROPROB"
        a = sim.get_amplitudes()
        assert a[0] == 1 and np.count_nonzero(a) == 1


def test_create_limits(qs):
    """A register whose state cannot be allocated is refused with ENOMEM
    (36 qubits of complex128: 1 TiB, more than the device holds), sizes
    outside 1..36 with EINVAL; the device stays usable."""
    with pytest.raises(qs.QsimError) as e:
        qs.Simulator(36, precision="c128", torch_memory=False)
    assert e.value.status == "ENOMEM"
    for bad in (0, 37, 40):
        with pytest.raises(qs.QsimError) as e:
            qs.Simulator(bad, precision="c64", torch_memory=False)
        assert e.value.status == "EINVAL"
    with make(qs, 4, "c128") as sim:
        sim.apply(np.array([[0, 1], [1, 0]], dtype=np.complex128), [2])
        a = sim.get_amplitudes()
    assert a[4] == 1 and np.count_nonzero(a) == 1

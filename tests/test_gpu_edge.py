"""Degenerate and boundary cases against the oracle: registers of 1-3 qubits
(plain and fused), gates controlled by every other qubit (two amplitudes
touched), a permutation of the whole register, diagonal-only circuits, empty
queues, empty term lists and zero-length reads."""
import math

import numpy as np
import pytest

import circuitgen as cg
from helpers import TOL64_INFID, infidelity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1612_08091_gb300 as q

    q.load()
    return q


def random_ops(n, count, seed):
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(count):
        kind = rng.integers(0, 5 if n >= 2 else 2)
        q = [int(v) for v in rng.permutation(n)]
        if kind == 0:
            ops.append(cg.op("U3", (q[0],), (), tuple(rng.uniform(0, 2 * math.pi, 3))))
        elif kind == 1:
            ops.append(cg.op("RZ", (q[0],), (), (float(rng.uniform(0, 2 * math.pi)),)))
        elif kind == 2:
            ops.append(cg.op("X", (q[0],), (q[1],)))
        elif kind == 3:
            ops.append(cg.op("Z", (q[0],), (q[1],)))
        else:
            t = min(n, 3)
            ops.append(cg.op("MAT", tuple(q[:t]), (), (cg.random_unitary(1 << t, int(rng.integers(1 << 30))),)))
    return ops


def random_terms(n, count, seed):
    rng = np.random.default_rng(seed)
    full = (1 << n) - 1
    return [(float(rng.uniform(-1, 1)), int(rng.integers(0, full + 1)), int(rng.integers(0, full + 1)))
            for _ in range(count)]


def check(prec, got, want):
    if prec == "c128":
        assert np.max(np.abs(got - want)) <= 1e-12
    else:
        assert infidelity(want, got) <= TOL64_INFID
        assert np.max(np.abs(got - want)) <= 1e-5


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("fusion", ["none", "greedy"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_registers(qs, oracle_mod, prec, fusion, n):
    ops = random_ops(n, 12, seed=n * 10 + (fusion == "greedy"))
    terms = random_terms(n, 5, seed=n)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    tol = 1e-12 if prec == "c128" else 1e-5
    with qs.Simulator(n, precision=prec, fusion=fusion) as sim:
        sim.flush()  # nothing queued
        sim.run(ops)
        got = sim.get_amplitudes()
        check(prec, got, ref.psi)
        p1, nrm = sim.probs_all()
        np.testing.assert_allclose(p1, ref.probs_all(), atol=tol)
        assert abs(nrm - 1.0) <= tol
        assert abs(sim.expect(terms) - ref.expect(terms)) <= 10 * tol
        assert sim.expect([]) == 0.0
        assert len(sim.get_amplitudes(1 << n, 0)) == 0
        u = 0.6180339887
        j = sim.measure_all(u)
        c = np.cumsum(np.abs(ref.psi) ** 2)
        jr = int(np.searchsorted(c, u * c[-1], side="right"))
        assert j == jr or abs(c[min(j, jr)] - u * c[-1]) < 1e-6
        after = sim.get_amplitudes()
        assert abs(abs(after[j]) - 1.0) <= tol and np.sum(np.abs(after) ** 2) - abs(after[j]) ** 2 <= tol


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [5, 14])
def test_gates_controlled_by_every_other_qubit(qs, oracle_mod, prec, n):
    psi = cg.random_state(n, seed=n + 1)
    rng = np.random.default_rng(n)
    ops = []
    for t in (0, n - 1, n // 2):
        ctl = tuple(q for q in range(n) if q != t)
        ops += [cg.op("Z", (t,), ctl), cg.op("X", (t,), ctl),
                cg.op("U3", (t,), ctl, tuple(rng.uniform(0, 2 * math.pi, 3))),
                cg.op("R", (t,), ctl, (float(rng.uniform(0, 2 * math.pi)),))]
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec) as sim:
        sim.set_amplitudes(psi)
        sim.run(ops)
        got = sim.get_amplitudes()
    # only the amplitudes with all controls set change
    check(prec, got, ref.psi)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_permutation_of_the_whole_register(qs, oracle_mod, prec):
    n = 6
    perm = np.random.default_rng(4).permutation(1 << n)
    qubits = (3, 0, 5, 1, 4, 2)
    psi = cg.random_state(n, seed=12)
    ref = oracle_mod.OracleSim(n, psi=psi)
    ref.apply_permutation(perm, qubits, ())
    with qs.Simulator(n, precision=prec) as sim:
        sim.set_amplitudes(psi)
        sim.apply_permutation(perm, qubits, ())
        got = sim.get_amplitudes()
    np.testing.assert_allclose(got, ref.psi, atol=0 if prec == "c128" else 1e-7)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [2, 3, 13])
def test_diagonal_only_circuits(qs, oracle_mod, prec, n):
    rng = np.random.default_rng(n + 50)
    ops = []
    for _ in range(30):
        a, b = (int(v) for v in rng.permutation(n)[:2])
        k = rng.integers(0, 3)
        if k == 0:
            ops.append(cg.op("RZ", (a,), (), (float(rng.uniform(0, 6.28)),)))
        elif k == 1:
            ops.append(cg.op("R", (a,), (b,), (float(rng.uniform(0, 6.28)),)))
        else:
            ops.append(cg.op("Z", (a,), (b,)))
    psi = cg.random_state(n, seed=n)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec, fusion="greedy") as sim:
        sim.set_amplitudes(psi)
        sim.run(ops)
        got = sim.get_amplitudes()
        st = sim.stats()
    check(prec, got, ref.psi)
    assert st["passes"] < len(ops)

"""A register split into 2 or 4 shards held as libqsim handles on one GPU,
against the oracle: gates on local and global qubits (the exchange step runs
sim_swap_halves), probabilities, Pauli sums, measurement (sim_project with
the scale summed over shards) and full-register sampling."""
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


def brickwork_and_mixed(n, seed):
    """The benchmark brickwork (every qubit, CNOTs across the shard
    boundary) plus multi-qubit unitaries and controlled gates on random
    qubits."""
    rng = np.random.default_rng(seed)
    ops = cg.random_u3_brickwork(n, 4, seed)
    for k in range(12):
        qs_ = [int(v) for v in rng.permutation(n)]
        if k % 3 == 0:
            ops.append(cg.op("MAT", tuple(qs_[:3]), (), (cg.random_unitary(8, seed + k),)))
        elif k % 3 == 1:
            ops.append(cg.op("U3", (qs_[0],), (qs_[1], qs_[2]), tuple(rng.uniform(0, 2 * np.pi, 3))))
        else:
            ops.append(cg.op("X", (qs_[0],), (qs_[1],)))
    return ops


@pytest.mark.parametrize("g", [1, 2])
@pytest.mark.parametrize("prec,fusion", [("c128", "none"), ("c64", "greedy")])
def test_sharded_register_against_oracle(qs, oracle_mod, g, prec, fusion):
    from paper_1612_08091_gb300.sharded import ShardedSimulator

    n = 18
    ops = brickwork_and_mixed(n, seed=31 + g)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    terms = cg.tfim_terms(n) + [(0.5, (1 << (n - 1)) | 1, 1 << 3)]
    tol = 1e-11 if prec == "c128" else 1e-5
    with ShardedSimulator(n, global_qubits=g, precision=prec, fusion=fusion) as sim:
        sim.run(ops)
        sim.flush()
        assert sim.exchanges > 0
        p1, nrm = sim.probs_all()
        np.testing.assert_allclose(p1, ref.probs_all(), atol=tol)
        assert abs(nrm - 1.0) <= tol
        assert abs(sim.expect(terms) - ref.expect(terms)) <= tol * sum(abs(c) for c, _, _ in terms)
        got = sim.get_amplitudes()
        if prec == "c128":
            assert np.max(np.abs(got - ref.psi)) <= 1e-11
        else:
            assert infidelity(ref.psi, got) <= TOL64_INFID
        # measure a global and a local qubit, then sample the register
        for q, u in ((n - 1, 0.3), (2, 0.7)):
            b, p = sim.measure(q, u)
            p1q = ref.probs_all()[q]
            assert b == ref.measure(q, u)
            assert abs(p - (p1q if b else 1.0 - p1q)) <= tol
        got = sim.get_amplitudes()
        if prec == "c128":
            assert np.max(np.abs(got - ref.psi)) <= 1e-11
        else:
            assert infidelity(ref.psi, got) <= TOL64_INFID
        sim.run(ops[:n])
        oracle_mod.run_ops(ref, ops[:n])
        u = 0.5772156649
        c = np.cumsum(np.abs(ref.psi) ** 2)  # before the oracle's collapse
        j = sim.measure_all(u)
        jr = ref.measure_all(u)
        if j != jr:
            # neighbouring outcomes where u * norm lies on their boundary
            assert abs(j - jr) == 1, (j, jr)
            assert abs(c[min(j, jr)] - u * c[-1]) < (1e-12 if prec == "c128" else 1e-6)
        after = sim.get_amplitudes()
        assert abs(abs(after[j]) - 1.0) <= tol and np.count_nonzero(after) == 1


def test_swap_halves_and_project_calls(qs, oracle_mod):
    """The two device calls of the exchange step, on their own."""
    n = 12
    a_psi, b_psi = cg.random_state(n, seed=1), cg.random_state(n, seed=2)
    with qs.Simulator(n, precision="c128") as a, qs.Simulator(n, precision="c128") as b:
        a.set_amplitudes(a_psi)
        b.set_amplitudes(b_psi)
        for qubit in (0, 5, n - 1):
            a.swap_halves(b, qubit)
            va, vb = a_psi.reshape(-1, 2, 1 << qubit), b_psi.reshape(-1, 2, 1 << qubit)
            tmp = va[:, 1, :].copy()
            va[:, 1, :] = vb[:, 0, :]
            vb[:, 0, :] = tmp
            np.testing.assert_array_equal(a.get_amplitudes(), a_psi)
            np.testing.assert_array_equal(b.get_amplitudes(), b_psi)
        a.project([3, 7], [1, 0], 2.0)
        idx = np.arange(1 << n)
        keep = (((idx >> 3) & 1) == 1) & (((idx >> 7) & 1) == 0)
        want = np.where(keep, 2.0 * a_psi, 0.0)
        np.testing.assert_array_equal(a.get_amplitudes(), want)
        a.project([], [], 0.0)
        assert not np.any(a.get_amplitudes())
        with pytest.raises(qs.QsimError) as e:
            a.swap_halves(a, 0)
        assert e.value.status == "EINVAL"
        with qs.Simulator(n - 1, precision="c128") as c:
            with pytest.raises(qs.QsimError):
                a.swap_halves(c, 0)


def test_sharded_c64_long_circuit_keeps_the_norm(qs, oracle_mod):
    """A depth-40 brickwork on 2 shards of a 20-qubit complex64 register,
    flushed after every layer so that the top qubit is exchanged in every
    layer (some 40 exchanges; unflushed, the scheduler needs only a few).
    Each exchange passes the shards' exact norms on to their block passes'
    norm control, so the norm stays at 1 instead of taking a new, slightly
    drifted target after every exchange."""
    from paper_1612_08091_gb300.sharded import ShardedSimulator

    n = 20
    ops = cg.random_u3_brickwork(n, 40, seed=8091)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with ShardedSimulator(n, global_qubits=1, precision="c64", fusion="greedy") as sim:
        k = 0
        for layer in range(40):
            cnt = n + len(range(layer % 2, n - 1, 2))
            sim.run(ops[k:k + cnt])
            sim.flush()
            k += cnt
        assert k == len(ops)
        p1, nrm = sim.probs_all()
        ex = sim.exchanges
        got = sim.get_amplitudes()
    print("sharded c64, 20 qubits depth 40: %d exchanges, |norm2-1| %.2e, infidelity %.2e"
          % (ex, abs(nrm - 1.0), infidelity(ref.psi, got)))
    assert ex >= 20
    assert abs(nrm - 1.0) <= 2e-6
    assert infidelity(ref.psi, got) <= TOL64_INFID
    np.testing.assert_allclose(p1, ref.probs_all(), atol=1e-5)

"""6-qubit tensor-core blocks (complex64, tcgen05 with the state operand in
tensor memory, BF16x3) against the oracle.

Gates act on at most 5 qubits, so a 6-qubit block is made of overlapping
random unitaries on subsets of S (5 + 5 + 2 qubits covering all of S); with
kmax 6 the greedy planner multiplies them into one 64 x 64 block."""
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


def six_block_ops(S, seed):
    S = tuple(S)
    return [cg.op("MAT", S[:5], (), (cg.random_unitary(32, seed),)),
            cg.op("MAT", S[1:], (), (cg.random_unitary(32, seed + 1),)),
            cg.op("MAT", (S[5], S[0]), (), (cg.random_unitary(4, seed + 2),))]


PLACEMENTS = [
    (13, (0, 1, 2, 3, 4, 5)),        # lowest qubits (rows pair up), one tile
    (13, (7, 8, 9, 10, 11, 12)),     # highest
    (14, (1, 2, 3, 4, 5, 6)),        # low, without qubit 0
    (15, (0, 3, 6, 9, 12, 14)),      # spread, with qubit 0
    (16, (2, 5, 6, 7, 13, 15)),      # spread, without qubit 0
    (17, (16, 0, 9, 4, 12, 1)),      # unsorted target order
    (16, (0, 1, 2, 3, 4, 9)),        # qubits 0..3 (quad fragments), 8 tiles
    (17, (3, 0, 12, 2, 1, 5)),       # qubits 0..3, unsorted, 16 tiles
]


@pytest.mark.parametrize("n,S", PLACEMENTS)
@pytest.mark.parametrize("terms", [3, 5])
def test_six_qubit_block_placements(qs, oracle_mod, n, S, terms):
    psi = cg.random_state(n, seed=n * 11 + sum(S))
    ops = six_block_ops(S, seed=3 * sum(S) + n)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=6, tc_terms=terms) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
        st = sim.stats()
    assert kt.get("block_tc6", {}).get("launches", 0) == 1, kt
    assert st["passes"] == 1
    inf = infidelity(ref.psi, got)
    assert inf <= (1e-7 if terms == 5 else TOL64_INFID), inf
    assert np.max(np.abs(got - ref.psi)) <= (2e-4 if terms == 3 else 2e-5)


def test_kmax6_long_circuit_accuracy(qs, oracle_mod):
    """Depth-40 brickwork on 20 qubits: fewer passes than with 5-qubit blocks,
    the same accuracy bar, norm drift held by the tracking."""
    n = 20
    ops = cg.random_u3_brickwork(n, 40, seed=8091)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    terms_zz = cg.zz_chain_terms(n)
    e_ref = ref.expect(terms_zz)
    passes = {}
    for kmax in (5, 6):
        with qs.Simulator(n, precision="c64", fusion="greedy", kmax=kmax) as sim:
            sim.set_profiling(True)
            sim.run(ops)
            got = sim.get_amplitudes()
            st = sim.stats()
            kt = sim.kernel_times()
            e = sim.expect(terms_zz)
        passes[kmax] = st["passes"]
        inf = infidelity(ref.psi, got)
        drift = abs(np.vdot(got, got).real - 1.0)
        print("n=20 depth 40, kmax %d: %d passes (%s), infidelity %.3e, |norm-1| %.3e, <ZZ> error %.3e"
              % (kmax, st["passes"], {k: v["launches"] for k, v in kt.items()}, inf, drift, abs(e - e_ref)))
        assert inf <= TOL64_INFID
        assert drift <= 5e-6
        assert abs(e - e_ref) <= 1e-5 * len(terms_zz)
        if kmax == 6:
            assert kt.get("block_tc6", {}).get("launches", 0) > 0, kt
    assert passes[6] < passes[5]


@pytest.mark.parametrize("kmax", [5, 6])
def test_kmax5_and_6_against_oracle(qs, oracle_mod, kmax):
    n = 22
    ops = cg.random_u3_brickwork(n, 8, seed=17) + cg.qft_ops(n)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=kmax) as a:
        a.set_profiling(True)
        a.run(ops)
        got = a.get_amplitudes()
        kt = a.kernel_times()
    assert kt.get("block_tc6" if kmax == 6 else "block_tc", {}).get("launches", 0) > 0, kt
    assert infidelity(ref.psi, got) <= TOL64_INFID


@pytest.mark.parametrize("prec,n,tensor_cores", [("c128", 14, True), ("c64", 12, True), ("c64", 14, False)])
def test_kmax6_falls_back_to_five(qs, oracle_mod, prec, n, tensor_cores):
    """kmax 6 where no 6-qubit executor exists (complex128, fewer than 13
    qubits, tensor cores off) plans blocks of at most 5 qubits."""
    S = tuple(range(n - 6, n))
    ops = six_block_ops(S, seed=n)
    psi = cg.random_state(n, seed=5)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec, fusion="greedy", kmax=6, tensor_cores=tensor_cores) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
    assert "block_tc6" not in kt or kt["block_tc6"]["launches"] == 0, kt
    if prec == "c128":
        assert np.max(np.abs(got - ref.psi)) <= 1e-11
    else:
        assert infidelity(ref.psi, got) <= TOL64_INFID


def test_kmax_outside_range_rejected(qs):
    for bad in (0, 7):
        with qs.Simulator(13, precision="c64") as sim:
            with pytest.raises(qs.QsimError) as e:
                sim.set_fusion("greedy", bad)
            assert e.value.status == "EINVAL"

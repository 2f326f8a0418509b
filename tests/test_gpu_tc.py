"""Tensor-core fused blocks (complex64, tcgen05, BF16x3) against the oracle.

Two random unitaries on the same qubit set S make one fused block, so these
cases run the block kernel for every kind of placement of S: the lowest
qubits, the highest, and mixed; 4-qubit blocks are padded to 5."""
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


def two_block_ops(S, seed):
    d = 1 << len(S)
    return [cg.op("MAT", S, (), (cg.random_unitary(d, seed),)), cg.op("MAT", S, (), (cg.random_unitary(d, seed + 1),))]


PLACEMENTS = [
    (12, (0, 1, 2, 3, 4)),        # lowest qubits, one tile
    (12, (7, 8, 9, 10, 11)),      # highest
    (13, (0, 3, 6, 9, 12)),       # spread
    (14, (2, 5, 6, 7, 13)),
    (16, (11, 12, 13, 14, 15)),
    (16, (0, 1, 14, 8, 3)),       # unsorted target order
    (15, (4, 5, 6, 7)),           # 4 qubits, padded to 5
    (14, (13, 0, 7)),             # 3 qubits: CUDA-core block
    (15, (0, 1, 2, 3, 10)),       # qubits 0..3 (quad fragments), 8 tiles
    (14, (2, 0, 3, 1)),           # 4 qubits padded to {0..4}: quad fragments
]


@pytest.mark.parametrize("n,S", PLACEMENTS)
@pytest.mark.parametrize("terms", [3, 5])
def test_fused_block_placements(qs, oracle_mod, n, S, terms):
    psi = cg.random_state(n, seed=n * 7 + len(S))
    ops = two_block_ops(S, seed=sum(S) + n)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", tc_terms=terms) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
    if len(S) >= 4:
        assert kt.get("block_tc", {}).get("launches", 0) == 1, kt
    inf = infidelity(ref.psi, got)
    assert inf <= (1e-7 if terms == 5 else TOL64_INFID), inf
    assert np.max(np.abs(got - ref.psi)) <= (2e-4 if terms == 3 else 2e-5)


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_tc_and_cuda_core_blocks_against_oracle(qs, oracle_mod, tensor_cores):
    n = 18
    ops = cg.random_u3_brickwork(n, 6, seed=5)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=5, tensor_cores=tensor_cores) as a:
        a.set_profiling(True)
        a.run(ops)
        got = a.get_amplitudes()
        kt = a.kernel_times()
    assert kt.get("block_tc" if tensor_cores else "block_dense", {}).get("launches", 0) > 0, kt
    assert infidelity(ref.psi, got) <= TOL64_INFID


def test_tc_long_circuit_accuracy(qs, oracle_mod):
    n = 20
    ops = cg.random_u3_brickwork(n, 40, seed=8091)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    terms_zz = cg.zz_chain_terms(n)
    e_ref = ref.expect(terms_zz)
    rows = []
    for terms in (3, 5):
        for track in (True, False):
            with qs.Simulator(n, precision="c64", fusion="greedy", tc_terms=terms, norm_tracking=track) as sim:
                sim.run(ops)
                got = sim.get_amplitudes()
                st = sim.stats()
                e = sim.expect(terms_zz)
            inf = infidelity(ref.psi, got)
            drift = abs(np.vdot(got, got).real - 1.0)
            rows.append((terms, track, inf, drift, abs(e - e_ref)))
            print("n=20 depth 40, %d products, norm tracking %s: %d passes, infidelity %.3e, |norm-1| %.3e, "
                  "<ZZ> error %.3e" % (terms, track, st["passes"], inf, drift, abs(e - e_ref)))
    for terms, track, inf, drift, eerr in rows:
        assert inf <= TOL64_INFID
        if track:
            # every block pass scales its output back to the norm target
            assert drift <= 2e-6
            assert eerr <= 1e-5 * len(terms_zz)

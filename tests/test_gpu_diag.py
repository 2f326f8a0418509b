"""Diagonal blocks: runs of commuting diagonal gates (controlled phases of the
QFT, the controlled z-rotation chain of the paper's benchmark circuit, Z/S/T/
RZ layers) merged into one multiply-by-table pass, against the oracle."""
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


def diag_layer_ops(n, seed):
    """Only diagonal gates (applied to a random state): RZ, T, CZ pairs, a
    two-target diagonal matrix and a multi-controlled Z."""
    rng = np.random.default_rng(seed)
    ops = []
    for q in range(n):
        ops.append(cg.op("RZ", (q,), (), (float(rng.uniform(0, 6.28)),)))
        ops.append(cg.op("T", (q,)))
    for q in range(0, n - 1, 2):
        ops.append(cg.op("Z", (q + 1,), (q,)))
    ops.append(cg.op("MAT", (3, 0), (), (np.diag(np.exp(1j * rng.uniform(0, 6.28, 4))),)))
    ops.append(cg.op("Z", (n - 1,), (0, 5, 9)))
    return ops


CIRCUITS = {
    "qft": lambda n: cg.basis_prep_ops(12345 % (1 << n), n) + cg.qft_ops(n),
    "hcrz": lambda n: cg.hadamard_crz_chain(n, seed=7),
    "layers": lambda n: diag_layer_ops(n, seed=3),
}


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_diag_blocks_match_oracle(qs, oracle_mod, prec, name):
    n = 16
    ops = CIRCUITS[name](n)
    psi = cg.random_state(n, seed=5) if name == "layers" else None
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec, fusion="greedy") as sim:
        if psi is not None:
            sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
        st = sim.stats()
    assert kt.get("block_diag", {}).get("launches", 0) >= 1, kt
    if prec == "c128":
        assert np.max(np.abs(got - ref.psi)) <= 1e-11
    else:
        assert infidelity(ref.psi, got) <= TOL64_INFID
    print("%s %s: %d gates in %d passes, %d diagonal blocks" % (name, prec, len(ops), st["passes"],
                                                                 kt["block_diag"]["launches"]))


def test_diag_block_c128_double_float(qs, oracle_mod):
    n = 14
    ops = cg.hadamard_crz_chain(n, seed=9)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c128", fusion="greedy", c128_df=True) as sim:
        sim.run(ops)
        got = sim.get_amplitudes()
    assert np.max(np.abs(got - ref.psi)) <= 1e-11

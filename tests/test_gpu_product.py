"""Product passes (layers of Hadamard-like one-qubit gates between gates
too wide for a block, applied 12 qubits per pass) against the oracle: the
greedy planner forms them on complex64 registers of 12 or more qubits;
every placement of the pass's qubits (below the tile, above it, both in one
pass) and every sign pattern; layers of general gates stay with the
blocks; Grover's search against its closed form with the norm held by the
norm control across all its product passes."""
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


def layered(n, wires, seed, layers=3):
    """Layers of Hadamard-like one-qubit gates on `wires` (each wire: an H
    with X before and after at random, so every sign pattern of the
    butterfly occurs), each followed by a Z on qubit n-1 controlled by all
    others (a gate no block can take)."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(layers):
        for w in wires:
            if rng.integers(0, 2):
                ops.append(cg.op("X", (w,)))
            ops.append(cg.op("H", (w,)))
            if rng.integers(0, 2):
                ops.append(cg.op("X", (w,)))
        ops.append(cg.op("Z", (n - 1,), tuple(range(n - 1))))
    return ops


CASES = [
    (12, tuple(range(12))),                          # one tile: every qubit in one pass
    (16, tuple(range(16))),                          # a low pass and a high pass
    (16, (0, 3, 5, 7, 9, 11, 2)),                    # only qubits below the tile
    (21, tuple(range(12, 21))),                      # only qubits above it: 8 + 1, runs of 16 and 2^11
    (21, (0, 1, 2) + tuple(range(12, 21))),          # low qubits folded into the last high pass
    (22, (1, 4, 6, 8, 10, 11, 13, 15, 16, 18, 19, 20, 21)),  # low pass and one high pass
    (13, (0, 1, 2, 3, 4, 5, 12)),                    # one pass, the top qubit folded with the low ones, 2 tiles
]


@pytest.mark.parametrize("n,wires", CASES)
def test_product_passes_against_oracle(qs, oracle_mod, n, wires):
    psi = cg.random_state(n, seed=7 * n + len(wires))
    ops = layered(n, wires, seed=n * 31 + sum(wires))
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=6) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
        p1, nrm = sim.probs_all()
    assert kt.get("product", {}).get("launches", 0) >= 1, kt
    # FP32 arithmetic on every gate (no bf16 split): far inside the 1e-5 bar
    inf = infidelity(ref.psi, got)
    assert inf <= 1e-9, inf
    assert np.max(np.abs(got - ref.psi)) <= 2e-6 * max(1.0, math.sqrt(len(ops) / 10.0))
    np.testing.assert_allclose(p1, ref.probs_all(), atol=1e-5)
    assert abs(nrm - 1.0) <= 1e-5


def test_product_passes_off_gives_blocks(qs, oracle_mod):
    """The same circuit with product passes disabled runs as 6-qubit blocks
    and agrees with the oracle too (the two paths compared with the oracle,
    not with each other)."""
    n = 16
    psi = cg.random_state(n, seed=3)
    ops = layered(n, tuple(range(n)), seed=4)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    for prod in (True, False):
        with qs.Simulator(n, precision="c64", fusion="greedy", kmax=6, product_passes=prod) as sim:
            sim.set_amplitudes(psi)
            sim.set_profiling(True)
            sim.run(ops)
            got = sim.get_amplitudes()
            kt = sim.kernel_times()
        assert ("product" in kt) == prod, kt
        assert infidelity(ref.psi, got) <= TOL64_INFID


def test_general_layers_stay_with_blocks(qs, oracle_mod):
    """A layer of U3 gates between the wide gates is no butterfly product:
    it runs as tensor-core blocks (general 2x2 factors would make a
    12-qubit product pass arithmetic-bound)."""
    n = 16
    rng = np.random.default_rng(11)
    ops = []
    for _ in range(2):
        ops += [cg.op("U3", (w,), (), tuple(rng.uniform(0, 2 * np.pi, 3))) for w in range(n)]
        ops.append(cg.op("Z", (n - 1,), tuple(range(n - 1))))
    psi = cg.random_state(n, seed=12)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=6) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
    assert "product" not in kt and kt.get("block_tc6", {}).get("launches", 0) >= 4, kt
    assert infidelity(ref.psi, got) <= TOL64_INFID


def test_grover_search_with_product_passes(qs):
    """Grover's full search on 16 qubits (r = 201 iterations, 2 product
    items of 2 passes each per iteration): the marked amplitude against the
    closed form (-1)^r sin((2r + 1) theta), the norm held at 1.  Without the
    norm control the FP32 Hadamard entries alone (fl(1/sqrt 2) is 1.7e-8
    small) would shrink the norm by 5.5e-7 per layer of 16 wires, 2.2e-4 over
    the 403 layers."""
    n = 16
    marked = int(cg.grover_marked(n, 2017)) & ((1 << n) - 1)
    r = cg.grover_iterations(n)
    ops = cg.grover_ops(n, marked, iterations=r)
    theta = math.asin(2.0 ** (-n / 2))
    want = (-1) ** r * math.sin((2 * r + 1) * theta)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=6) as sim:
        sim.set_profiling(True)
        sim.run(ops)
        sim.flush()
        a = sim.get_amplitudes(marked, 1)[0]
        p1, nrm = sim.probs_all()
        kt = sim.kernel_times()
    # one timed entry per product item (two per iteration, each 2 passes)
    assert kt["product"]["launches"] >= 2 * r, kt
    assert abs(a - want) <= 1e-5, (a, want)
    assert abs(abs(a) ** 2 - math.sin((2 * r + 1) * theta) ** 2) <= 1e-5
    assert abs(nrm - 1.0) <= 1e-6, nrm


def test_product_and_block_passes_share_the_norm_chain(qs, oracle_mod):
    """Product passes and tensor-core block passes alternate in one norm
    chain: H / X layers between many-controlled Z gates, then a U3 + CNOT
    brickwork segment (blocks), repeated; the state against the oracle and
    the raw norm at 1."""
    n = 18
    ops = []
    for rep in range(3):
        ops += layered(n, tuple(range(n)), seed=100 + rep, layers=2)
        bw = cg.random_u3_brickwork(n, 3, seed=200 + rep)
        ops += bw
        ops.append(cg.op("Z", (n - 1,), tuple(range(n - 1))))
    psi = cg.random_state(n, seed=22)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c64", fusion="greedy", kmax=6) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
        p1, nrm = sim.probs_all()
    assert kt.get("product", {}).get("launches", 0) >= 3 and kt.get("block_tc6", {}).get("launches", 0) >= 3, kt
    assert infidelity(ref.psi, got) <= TOL64_INFID
    np.testing.assert_allclose(p1, ref.probs_all(), atol=1e-5)
    assert abs(nrm - 1.0) <= 1e-5, nrm

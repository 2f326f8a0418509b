"""Permutation blocks: runs of permutation gates (X with controls, Toffoli,
SWAP) planned into one pass of the emulated-permutation kernels, against the
oracle and the adder's closed form."""
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


def perm_launches(kt):
    return sum(kt.get(c, {}).get("launches", 0) for c in ("permute", "permute_cycles", "permute_cycles_bulk"))


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_adder_closed_form_and_oracle(qs, oracle_mod, prec):
    m = 9
    n = 2 * m + 2
    ops = cg.ripple_adder_ops(m, reps=2)
    # a superposition over a few basis inputs: each goes to a + 2b
    rng = np.random.default_rng(4)
    inputs = [(int(a), int(b)) for a, b in rng.integers(0, 1 << m, (4, 2))]
    psi = np.zeros(1 << n, dtype=np.complex128)
    amps = cg.random_state(2, seed=1)
    for (a, b), z in zip(inputs, amps):
        psi[cg.adder_basis_index(m, a, b)] = z
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec, fusion="greedy") as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
        st = sim.stats()
    assert perm_launches(kt) > 0, kt
    assert st["passes"] < len(ops) / 5
    # complex128: amplitudes only move; complex64: a dense tensor-core block
    # (BF16x3) may take part of the circuit
    tol = 0 if prec == "c128" else 1e-5
    assert np.max(np.abs(got - ref.psi)) <= tol
    for (a, b), z in zip(inputs, amps):
        s1 = (a + b) % (1 << m)
        c1 = (a + b) >> m
        s2 = (a + s1) % (1 << m)
        c2 = c1 ^ ((a + s1) >> m)
        assert abs(got[cg.adder_basis_index(m, a, s2, c2)] - z) <= max(tol, 1e-15)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("p_dense", [0.1, 0.4])
def test_mixed_permutation_heavy_circuits(qs, oracle_mod, prec, p_dense):
    n = 16
    rng = np.random.default_rng(int(p_dense * 10) + (prec == "c64"))
    ops = []
    for _ in range(300):
        q = [int(v) for v in rng.permutation(n)[:3]]
        r = rng.random()
        if r < p_dense:
            ops.append(cg.op("U3", (q[0],), (), tuple(rng.uniform(0, 6.28, 3))))
        elif r < p_dense + 0.4 * (1 - p_dense):
            ops.append(cg.op("X", (q[0],), (q[1],)))
        elif r < p_dense + 0.8 * (1 - p_dense):
            ops.append(cg.op("X", (q[0],), (q[1], q[2])))
        else:
            ops.append(cg.op("SWAP", (q[0], q[1])))
    psi = cg.random_state(n, seed=17)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec, fusion="greedy") as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
    if p_dense < 0.2:
        assert perm_launches(kt) > 0, kt
    if prec == "c128":
        assert np.max(np.abs(got - ref.psi)) <= 1e-11
    else:
        assert infidelity(ref.psi, got) <= TOL64_INFID


def test_permutation_blocks_can_be_switched_off(qs):
    m = 6
    n = 2 * m + 2
    ops = cg.ripple_adder_ops(m, reps=3)
    out = {}
    for on in (True, False):
        with qs.Simulator(n, precision="c128", fusion="greedy", perm_blocks=on) as sim:
            sim.reset(cg.adder_basis_index(m, 21, 42))
            sim.set_profiling(True)
            sim.run(ops)
            out[on] = (sim.get_amplitudes(), perm_launches(sim.kernel_times()), sim.stats()["passes"])
    assert out[True][1] > 0 and out[False][1] == 0
    assert out[True][2] < out[False][2]
    np.testing.assert_array_equal(out[True][0], out[False][0])

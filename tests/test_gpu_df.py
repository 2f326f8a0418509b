"""complex128 with double-float gate arithmetic (qsim_opts.c128_double_float)
against the FP64 oracle: one-qubit dense, diagonal and phase gates at every
placement kind, multi-target dense gates, a 20-qubit depth-10 random circuit
plain and with fused blocks.  Bound: 1e-11 per amplitude, the same as the
FP64 plain path."""
import math

import numpy as np
import pytest

import circuitgen as cg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1612_08091_gb300 as q

    q.load()
    return q


CASES = [("U3", (0,), ()), ("U3", (13,), ()), ("U3", (5,), (0, 9)), ("RZ", (7,), ()), ("RZ", (2,), (11,)),
         ("R", (3,), (12,)), ("R", (0,), ()), ("Z", (13,), tuple(range(13))), ("H", (1,), ()), ("X", (4,), (6,))]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_df_single_gates(qs, oracle_mod, case):
    n = 14
    kind, t, c = CASES[case]
    rng = np.random.default_rng(case)
    if kind == "U3":
        op = cg.op(kind, t, c, tuple(rng.uniform(0, 2 * math.pi, 3)))
    elif kind in ("RZ", "R"):
        op = cg.op(kind, t, c, (float(rng.uniform(0, 2 * math.pi)),))
    else:
        op = cg.op(kind, t, c)
    psi = cg.random_state(n, seed=200 + case)
    ref = oracle_mod.OracleSim(n, psi=psi)
    ref.apply_op(op)
    with qs.Simulator(n, precision="c128", c128_df=True) as sim:
        sim.set_amplitudes(psi)
        sim.apply_op(op)
        got = sim.get_amplitudes()
    err = np.max(np.abs(got - ref.psi))
    assert err <= 1e-11, err
    # the error is that of ~47-bit arithmetic, not of FP32
    assert err <= 1e-13 * np.max(np.abs(ref.psi)) * 64


def test_df_random_circuit(qs, oracle_mod):
    n = 20
    ops = cg.random_u3_brickwork(n, 10, seed=8091)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c128", c128_df=True) as sim:
        sim.run(ops)
        got = sim.get_amplitudes()
    err = np.max(np.abs(got - ref.psi))
    print("20-qubit depth-10 double-float max error %.3e" % err)
    assert err <= 1e-11


@pytest.mark.parametrize("width,controls", [(2, ()), (3, (12,)), (4, ()), (5, ()), (5, (0, 13))])
def test_df_multi_target_gate(qs, oracle_mod, width, controls):
    """A k-target dense gate (random unitary) with the double-float block
    kernel, at spread and unsorted targets."""
    n = 14
    rng = np.random.default_rng(width * 7 + len(controls))
    free = [q for q in range(n) if q not in controls]
    targets = tuple(int(q) for q in rng.permutation(free)[:width])
    op = cg.op("MAT", targets, controls, (cg.random_unitary(1 << width, seed=width + 40),))
    psi = cg.random_state(n, seed=width + 3)
    ref = oracle_mod.OracleSim(n, psi=psi)
    oracle_mod.run_ops(ref, [op])
    with qs.Simulator(n, precision="c128", c128_df=True) as sim:
        sim.set_amplitudes(psi)
        sim.apply_op(op)
        got = sim.get_amplitudes()
    assert np.max(np.abs(got - ref.psi)) <= 1e-11


@pytest.mark.parametrize("kmax", [3, 5])
def test_df_fused_random_circuit(qs, oracle_mod, kmax):
    """Fused complex128 blocks (greedy, kmax 3 and 5) in double-float
    arithmetic on the 20-qubit depth-10 random circuit."""
    n = 20
    ops = cg.random_u3_brickwork(n, 10, seed=8091)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c128", fusion="greedy", kmax=kmax, c128_df=True) as sim:
        sim.set_profiling(True)
        sim.run(ops)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
        st = sim.stats()
    assert kt.get("block_dense", {}).get("launches", 0) > 0, kt
    assert st["passes"] < len(ops)
    err = np.max(np.abs(got - ref.psi))
    print("kmax %d: %d passes, max |amplitude error| %.3e" % (kmax, st["passes"], err))
    assert err <= 1e-11

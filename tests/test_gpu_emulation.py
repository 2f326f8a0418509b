"""Emulated classical functions on registers (the paper's BasicMathGate,
Sec. 4.3.3) against the oracle, and Shor's order finding for 7 mod 15 with
the semi-classical measure-and-reset loop of Appendix A.3."""
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


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("qubits,controls", [((0, 1, 2, 3), ()), ((13, 2, 7), (0,)), (tuple(range(4, 16)), ()),
                                             ((5, 9), (1, 3, 11))])
def test_permutation_matches_oracle(qs, oracle_mod, prec, qubits, controls):
    n = 16
    rng = np.random.default_rng(len(qubits) + 7 * len(controls))
    perm = rng.permutation(1 << len(qubits))
    psi = cg.random_state(n, seed=4)
    ref = oracle_mod.OracleSim(n, psi=psi)
    ref.apply_permutation(perm, qubits, controls)
    with qs.Simulator(n, precision=prec) as sim:
        sim.set_amplitudes(psi)
        sim.apply_permutation(perm, qubits, controls)
        got = sim.get_amplitudes()
    tol = 0 if prec == "c128" else 1e-7  # amplitudes only move (c64 storage rounding only)
    np.testing.assert_allclose(got, ref.psi, atol=tol)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["random", "add", "fixed_points", "identity"])
def test_permutation_cycle_walk(qs, oracle_mod, prec, kind):
    """A register above the lowest 4 KB of amplitudes (qubits 14..19 of 24,
    one control on qubit 22; 2^17 amplitudes per register value, so even one
    cycle makes 256 tasks of 4 KB) is permuted along the cycles of f in place:
    a random bijection (several cycles of mixed lengths), x -> x + 5 mod 64
    (one cycle), a bijection with fixed points, and the identity."""
    n, qubits, controls = 24, (16, 14, 19, 15, 18, 17), (22,)
    rng = np.random.default_rng(12)
    D = 1 << len(qubits)
    if kind == "random":
        perm = rng.permutation(D)
    elif kind == "add":
        perm = (np.arange(D) + 5) % D
    elif kind == "fixed_points":
        perm = np.arange(D)
        moved = rng.choice(D, 20, replace=False)
        perm[moved] = moved[rng.permutation(20)]
    else:
        perm = np.arange(D)
    psi = cg.random_state(n, seed=9)
    ref = oracle_mod.OracleSim(n, psi=psi)
    ref.apply_permutation(perm, qubits, controls)
    with qs.Simulator(n, precision=prec) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.apply_permutation(perm, qubits, controls)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
    if kind != "identity":
        walks = sum(kt.get(c, {}).get("launches", 0) for c in ("permute_cycles", "permute_cycles_bulk"))
        assert walks == 1, kt
    tol = 0 if prec == "c128" else 1e-7
    np.testing.assert_allclose(got, ref.psi, atol=tol)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["random", "add", "fixed_points"])
def test_permutation_bulk_copy_walk(qs, oracle_mod, prec, kind):
    """A register above the lowest 16 KB of amplitudes with enough 16 KB
    slices (qubits 16..21 of 27, one control on qubit 25: 2^20 amplitudes per
    register value) goes through the bulk-copy cycle walk."""
    n, qubits, controls = 27, (18, 16, 21, 17, 20, 19), (25,)
    rng = np.random.default_rng(13)
    D = 1 << len(qubits)
    if kind == "random":
        perm = rng.permutation(D)
    elif kind == "add":
        perm = (np.arange(D) + 11) % D
    else:
        perm = np.arange(D)
        moved = rng.choice(D, 9, replace=False)
        perm[moved] = moved[np.roll(np.arange(9), 1)]
    psi = cg.random_state(n, seed=10)
    ref = oracle_mod.OracleSim(n, psi=psi)
    ref.apply_permutation(perm, qubits, controls)
    with qs.Simulator(n, precision=prec) as sim:
        sim.set_amplitudes(psi)
        sim.set_profiling(True)
        sim.apply_permutation(perm, qubits, controls)
        got = sim.get_amplitudes()
        kt = sim.kernel_times()
    assert kt.get("permute_cycles_bulk", {}).get("launches", 0) == 1, kt
    tol = 0 if prec == "c128" else 1e-7
    assert np.max(np.abs(got - ref.psi)) <= tol


def test_permutation_tiled_when_register_is_low(qs):
    """The tiled kernel takes registers within the lowest 4 KB of amplitudes."""
    with qs.Simulator(16, precision="c64") as sim:
        sim.set_profiling(True)
        sim.apply_permutation(np.roll(np.arange(16), 3), (0, 1, 2, 3), ())
        kt = sim.kernel_times()
    assert kt.get("permute", {}).get("launches", 0) == 1 and "permute_cycles" not in kt, kt


def test_permutation_rejects_non_bijection(qs):
    with qs.Simulator(6) as sim:
        with pytest.raises(qs.QsimError) as e:
            sim.apply_permutation([0, 0, 1, 2], [0, 1])
        assert e.value.status == "EINVAL"


def shor_order_finding(sim, a, N, m, draws):
    """Register x on qubits 1..4 starts at |1>; qubit 0 is the recycled
    control.  Round k: H, controlled multiply-by a^(2^(m-1-k)) mod N (an
    emulated permutation: identity for x >= N), rotations conditioned on
    the earlier outcomes, H, measure, reset."""
    xq = [1, 2, 3, 4]
    sim.apply_op(cg.op("X", (1,)))
    bits = []
    for k in range(m):
        ak = pow(a, 1 << (m - 1 - k), N)
        perm = [(ak * x) % N if x < N else x for x in range(16)]
        sim.apply_op(cg.op("H", (0,)))
        sim.apply_permutation(perm, xq, (0,))
        for i in range(k):
            if bits[i]:
                sim.apply_op(cg.op("R", (0,), (), (-math.pi / (1 << (k - i)),)))
        sim.apply_op(cg.op("H", (0,)))
        b = sim.measure(0, draws[k])
        b = b[0] if isinstance(b, tuple) else b
        bits.append(b)
        if b:
            sim.apply_op(cg.op("X", (0,)))
    # bits come least significant first: phase = sum bits[k] 2^k / 2^m
    return sum(b << k for k, b in enumerate(bits))


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_shor_order_finding_7_mod_15(qs, oracle_mod, prec):
    a, N, m = 7, 15, 6
    seen = set()
    for trial in range(6):
        draws = cg.uniform_draws(500 + trial, m)
        ref = oracle_mod.OracleSim(5)
        want = shor_order_finding(ref, a, N, m, draws)
        with qs.Simulator(5, precision=prec) as sim:
            got = shor_order_finding(sim, a, N, m, draws)
        assert got == want
        # the order of 7 mod 15 is 4: the measured phase is s/4 exactly
        assert (got * 4) % (1 << m) == 0
        seen.add(got)
    assert len(seen) >= 2  # different draws reach different multiples of 2^m/4

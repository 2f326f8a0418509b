"""Measurement-conditioned loop (Appendix A.3 of the paper: semi-classical
inverse QFT with one recycled control qubit, rotations conditioned on the
earlier outcomes, measure, reset).  Here it estimates the phase phi of
R(2 pi phi) on its eigenstate |1>; for phi = k / 2^m the m outcomes spell k
exactly with probability 1.  GPU and oracle run the same loop; the outcomes
must agree bit for bit and the final states within the tolerances."""
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


def phase_estimation(sim, m, k, draws, spectators=()):
    """qubit 0: recycled control; qubit 1: eigenstate |1> of R(2 pi k/2^m);
    optional spectator qubits carry an unrelated state.  Returns the bits
    in the order measured: the highest power of U comes first, so the first
    outcome is the least significant bit of k."""
    phi = k / float(1 << m)
    sim.apply_op(cg.op("X", (1,)))
    for q, th in spectators:
        sim.apply_op(cg.op("RY", (q,), (), (th,)))
    bits = []
    for j in range(m):
        sim.apply_op(cg.op("H", (0,)))
        # controlled U^(2^(m-1-j)) = controlled R(2 pi phi 2^(m-1-j))
        sim.apply_op(cg.op("R", (1,), (0,), (2 * math.pi * phi * (1 << (m - 1 - j)),)))
        # semi-classical inverse QFT: rotations conditioned on earlier results
        for i in range(j):
            if bits[i]:
                sim.apply_op(cg.op("R", (0,), (), (-math.pi / (1 << (j - i)),)))
        sim.apply_op(cg.op("H", (0,)))
        b = sim.measure(0, draws[j])
        b = b[0] if isinstance(b, tuple) else b
        bits.append(b)
        if b:
            sim.apply_op(cg.op("X", (0,)))  # reset the control
    return bits


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("m,k", [(4, 11), (6, 37), (8, 200)])
def test_semiclassical_phase_estimation(qs, oracle_mod, prec, m, k):
    n = 5
    draws = cg.uniform_draws(31 + k, m)
    spectators = [(2, 0.3), (3, 1.9), (4, -0.7)]
    ref = oracle_mod.OracleSim(n)
    bits_ref = phase_estimation(ref, m, k, draws, spectators)
    with qs.Simulator(n, precision=prec) as sim:
        bits = phase_estimation(sim, m, k, draws, spectators)
        psi = sim.get_amplitudes()
    want = [(k >> j) & 1 for j in range(m)]
    assert bits_ref == want
    assert bits == want
    tol = 1e-12 if prec == "c128" else 1e-6
    np.testing.assert_allclose(psi, ref.psi, atol=tol)

"""Full-size checks at the register sizes of the benchmark configurations,
in the launch configuration bench.py times (fused complex64, greedy k <= 5;
plain complex128).  The oracle cannot hold these states in seconds, so the
checks use properties that hold at any size (U U^dag = 1, QFT and Grover
closed forms on sampled amplitudes, probabilities of 1/2, cumulative-sum
sampling against a host cumsum) plus one direct oracle comparison of the
full depth-40 circuit structure at 26 qubits."""
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


def _free():
    import torch

    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def qft_amplitudes(x, n, idx):
    N = 1 << n
    r = (np.uint64(x) * idx.astype(np.uint64)) % np.uint64(N)
    return np.exp(2j * np.pi * r.astype(np.float64) / N) / math.sqrt(N)


# per-amplitude bounds relative to the amplitude magnitude 2^-15: complex64
# blocks carry about 1e-6 relative error per amplitude after a few passes
# (infidelity ~1e-11); complex128 about 1e-14
@pytest.mark.parametrize("prec,fusion,rel", [("c64", "greedy", 1e-4), ("c128", "none", 1e-9)])
def test_qft30_closed_form(qs, prec, fusion, rel):
    n = 30
    x = cg.random_basis_state(n, seed=8091)
    idx = np.unique(np.concatenate([np.arange(64), (1 << n) - 1 - np.arange(64),
                                    np.random.default_rng(1).integers(0, 1 << n, 4096)]))
    with qs.Simulator(n, precision=prec, fusion=fusion) as sim:
        sim.run(cg.basis_prep_ops(x, n) + cg.qft_ops(n))
        p1, nrm = sim.probs_all()
        got = np.array([sim.get_amplitudes(int(i), 1)[0] for i in idx])
    want = qft_amplitudes(x, n, idx)
    err = np.max(np.abs(got - want)) / 2.0 ** (-n / 2)
    print("QFT-30 %s: max relative amplitude error %.3e" % (prec, err))
    assert err <= rel, err
    np.testing.assert_allclose(p1, 0.5, atol=1e-5 if prec == "c64" else 1e-12)
    assert abs(nrm - 1.0) <= (1e-5 if prec == "c64" else 1e-12)
    _free()


def test_random32_depth40_roundtrip_fused(qs):
    n = 32
    ops = cg.random_u3_brickwork(n, 40, seed=8091)
    with qs.Simulator(n, precision="c64", fusion="greedy") as sim:
        sim.run(ops)
        sim.flush()
        mid = sim.get_amplitudes(0, 4)
        sim.run(cg.inverse_ops(ops))
        a0 = sim.get_amplitudes(0, 1)[0]
        p1, nrm = sim.probs_all()
    assert abs(mid[0]) < 1e-3  # the forward circuit spread the state
    # fidelity with |0...0> after U U^dag
    assert 1.0 - abs(a0) ** 2 / nrm <= 2 * TOL64_INFID, 1.0 - abs(a0) ** 2 / nrm
    assert np.max(p1) <= 2 * TOL64_INFID
    _free()


def test_fig7_circuit_roundtrip_30(qs):
    """The paper's benchmark circuit (Fig. 7: H on all, a controlled-Rz
    chain, H on all) on 30 qubits, then its inverse, each flushed as one
    short queue: the planner tries both dense tie rules there and launches
    the one with fewer items (6 passes each way); U U^dag returns |0...0>."""
    n = 30
    ops = cg.hadamard_crz_chain(n, 1612)
    with qs.Simulator(n, precision="c64", fusion="greedy") as sim:
        sim.reset_stats()
        sim.run(ops)
        sim.flush()
        forward = sim.stats()["passes"]
        sim.run(cg.inverse_ops(ops))
        a0 = sim.get_amplitudes(0, 1)[0]
        p1, nrm = sim.probs_all()
    assert forward == 6, forward
    assert 1.0 - abs(a0) ** 2 / nrm <= 2 * TOL64_INFID, 1.0 - abs(a0) ** 2 / nrm
    assert np.max(p1) <= 2 * TOL64_INFID
    assert abs(nrm - 1.0) <= 1e-5
    _free()


@pytest.mark.parametrize("df", [False, True])
def test_random32_roundtrip_plain_c128(qs, df):
    """U U^dag on 32 qubits, complex128, one launch per gate, in FP64 and in
    double-float arithmetic (about 2^-45 relative per product)."""
    n = 32
    ops = cg.random_u3_brickwork(n, 3, seed=8091)
    with qs.Simulator(n, precision="c128", fusion="none", c128_df=df) as sim:
        sim.run(ops + cg.inverse_ops(ops))
        a0 = sim.get_amplitudes(0, 1)[0]
        p1, nrm = sim.probs_all()
    assert abs(abs(a0) - 1.0) <= 1e-12
    assert abs(nrm - 1.0) <= 1e-12 and np.max(p1) <= 1e-12
    _free()


@pytest.mark.parametrize("prec,fusion,df", [("c64", "greedy", False), ("c128", "none", False),
                                            ("c128", "none", True), ("c128", "greedy", True)])
def test_random26_depth40_against_oracle(qs, oracle_mod, prec, fusion, df):
    n = 26
    ops = cg.random_u3_brickwork(n, 40, seed=8091)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision=prec, fusion=fusion, c128_df=df) as sim:
        sim.run(ops)
        got = sim.get_amplitudes()
        p1, _ = sim.probs_all()
        e = sim.expect(cg.zz_chain_terms(n))
    inf = infidelity(ref.psi, got)
    if prec == "c128":
        assert np.max(np.abs(got - ref.psi)) <= 1e-11
        np.testing.assert_allclose(p1, ref.probs_all(), atol=1e-11)
        assert abs(e - ref.expect(cg.zz_chain_terms(n))) <= 1e-11 * (n - 1)
    else:
        assert inf <= TOL64_INFID, inf
    np.testing.assert_allclose(p1, ref.probs_all(), atol=1e-5)
    assert abs(e - ref.expect(cg.zz_chain_terms(n))) <= 1e-5 * (n - 1)
    _free()


@pytest.mark.parametrize("prec,fusion", [("c64", "greedy"), ("c128", "none")])
def test_grover28_truncated_closed_form(qs, prec, fusion):
    n = 28
    marked = cg.grover_marked(n, seed=2017)
    r = 12  # of the 12867 iterations; the closed form holds after any number
    with qs.Simulator(n, precision=prec, fusion=fusion) as sim:
        sim.run(cg.grover_ops(n, marked, iterations=r))
        am = sim.get_amplitudes(marked, 1)[0]
        others = sim.get_amplitudes(0, 64)
        p1, nrm = sim.probs_all()
    theta = math.asin(2.0 ** (-n / 2))
    sign = (-1) ** r
    a_m = sign * math.sin((2 * r + 1) * theta)
    a_o = sign * math.cos((2 * r + 1) * theta) / math.sqrt((1 << n) - 1)
    tol = 1e-6 if prec == "c64" else 1e-12
    rel = 1e-4 if prec == "c64" else 1e-9  # relative to the unmarked amplitude
    assert abs(am - a_m) <= tol
    mask = np.arange(64) != marked
    err = np.max(np.abs(others[mask] - a_o)) / abs(a_o)
    print("Grover-28 %s: marked error %.3e, unmarked relative error %.3e" % (prec, abs(am - a_m), err))
    assert err <= rel
    # P(q = 1) from the closed form
    want = np.array([((marked >> q) & 1) * a_m ** 2 + a_o ** 2 * ((1 << (n - 1)) - ((marked >> q) & 1))
                     for q in range(n)])
    np.testing.assert_allclose(p1, want, atol=10 * tol)
    _free()


def test_measure_all_30_against_host_cumsum(qs):
    """30-qubit complex64 register: the reductions, whose partial sums run
    in FP32 over runs of at most 32 terms before FP64 takes over, against
    FP64 sums on the host of the same (exactly widened) amplitudes; then
    measure-all against a host cumulative sum."""
    n = 30
    ops = cg.random_u3_brickwork(n, 2, seed=5)
    u = float(cg.uniform_draws(8092, 1)[0])
    zz = [(1.0, 0, (1 << i) | (1 << (i + 1))) for i in (0, 9, 10, 28)]
    with qs.Simulator(n, precision="c64", fusion="greedy") as sim:
        sim.run(ops)
        psi = sim.get_amplitudes()
        p1_gpu, nrm_gpu = sim.probs_all()
        pq_gpu = [sim.prob(q) for q in (0, 5, 29)]
        zz_gpu = [sim.expect([t]) for t in zz]
        j = sim.measure_all(u)
        after = sim.get_amplitudes(j, 1)[0]
        p1, nrm = sim.probs_all()
    w = (psi.real ** 2 + psi.imag ** 2)
    del psi
    # FP32 stage: a chain of at most 33 roundings (the |psi|^2 and 32 adds),
    # relative 33 * 2^-24 = 2.0e-6 at worst for every partial sum, so for the
    # total; FP64 beyond that
    bound = 2.5e-6
    nrm_host = float(np.sum(w))
    assert abs(nrm_gpu - nrm_host) <= bound * nrm_host
    for q in range(n):
        p_host = float(w.reshape(-1, 2, 1 << q)[:, 1, :].sum())
        assert abs(p1_gpu[q] - p_host) <= bound * p_host, (q, p1_gpu[q], p_host)
        if q in (0, 5, 29):
            assert abs(pq_gpu[(0, 5, 29).index(q)] - p_host) <= bound * p_host
    for (c, _, z), e in zip(zz, zz_gpu):
        i = z.bit_length() - 2
        v = w.reshape(-1, 2, 2, 1 << i)
        e_host = float(v[:, 0, 0, :].sum() - v[:, 0, 1, :].sum() - v[:, 1, 0, :].sum() + v[:, 1, 1, :].sum())
        assert abs(e - e_host) <= bound * nrm_host, (i, e, e_host)
    c = np.cumsum(w)
    jr = int(np.searchsorted(c, u * c[-1], side="right"))
    assert j == jr or abs(c[min(j, jr)] - u * c[-1]) < 1e-6 * c[-1]
    assert abs(abs(after) - 1.0) < 1e-6 and abs(nrm - 1.0) < 1e-6
    np.testing.assert_allclose(p1, [(j >> q) & 1 for q in range(n)], atol=1e-6)
    _free()

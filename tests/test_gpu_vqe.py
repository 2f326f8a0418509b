"""Batched variational sweep (one persistent launch, CUDA graph, autotuned
tiles) against the FP64 oracle: each energy is the oracle's
<psi| -sum Z_i Z_{i+1} - 0.7 sum X_i |psi> of the same ansatz circuit."""
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


def oracle_energy(oracle_mod, c, h=0.7):
    n = c["n"]
    s = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(s, cg.hea_ops(n, c["ry"], c["rz"]))
    return s.expect(cg.tfim_terms(n, h))


def tol(n):
    # 1e-5 times the operator 1-norm (n-1 ZZ terms + 0.7 n X terms)
    return 1e-5 * max(1.0, (n - 1) + 0.7 * n)


def test_small_batch_all_paths(qs, oracle_mod):
    # sizes chosen to cover shared-memory circuits and, with m = 12, the
    # global-memory path (n = 13..16)
    rng = np.random.default_rng(3)
    circuits = cg.hea_batch(40, seed=11, nmin=2, nmax=16, lmin=0, lmax=4)
    nq = [c["n"] for c in circuits]
    nl = [c["L"] for c in circuits]
    angles = qs.hea_angles(circuits)
    want = np.array([oracle_energy(oracle_mod, c) for c in circuits])
    with qs.Batch(nq, nl) as b:
        for threads, m in [(512, 14), (256, 12), (1024, 13), (512, 12)]:
            b.set_config(threads, m)
            got = b.run(angles)
            for i, c in enumerate(circuits):
                assert abs(got[i] - want[i]) <= tol(c["n"]), (threads, m, c["n"], got[i], want[i])
            got2 = b.run(angles)  # graph replay
            np.testing.assert_array_equal(got, got2)
    del rng


@pytest.mark.parametrize("scale", [0.5, 3.3])
def test_angles_outside_half_turn(qs, oracle_mod, scale):
    """Rotation angles scaled beyond [-pi, pi] (and within [-pi/2, pi/2]):
    every reduction of theta/2 by a multiple of pi/2 (quarter turns with
    their X Z and sign) and the RZ half-angle period, in the shared-memory
    and the global-memory circuits."""
    circuits = cg.hea_batch(24, seed=31, nmin=3, nmax=16, lmin=1, lmax=3)
    for c in circuits:
        c["ry"] = c["ry"] * scale
        c["rz"] = c["rz"] * scale
    nq = [c["n"] for c in circuits]
    nl = [c["L"] for c in circuits]
    angles = qs.hea_angles(circuits)
    want = np.array([oracle_energy(oracle_mod, c) for c in circuits])
    with qs.Batch(nq, nl) as b:
        for threads, m in [(256, 12), (512, 14)]:
            b.set_config(threads, m)
            got = b.run(angles)
            for i, c in enumerate(circuits):
                assert abs(got[i] - want[i]) <= tol(c["n"]), (threads, m, c["n"], got[i], want[i])


def test_largest_circuits(qs, oracle_mod):
    """21..24 qubits, the top of the accepted range: up to 12 qubits above
    the 2^12-amplitude chunks (a phase table of 4096 entries), and at 24 qubits
    tile runs of one amplitude (plain loads instead of bulk copies)."""
    circuits = cg.hea_batch(4, seed=77, nmin=21, nmax=21, lmin=1, lmax=2)
    for c, n in zip(circuits, (21, 22, 23, 24)):
        rng = np.random.default_rng(n)
        c["n"] = n
        c["ry"] = rng.uniform(-np.pi, np.pi, size=(c["L"], n))
        c["rz"] = rng.uniform(-np.pi, np.pi, size=(c["L"], n))
    nq = [c["n"] for c in circuits]
    nl = [c["L"] for c in circuits]
    angles = qs.hea_angles(circuits)
    want = np.array([oracle_energy(oracle_mod, c) for c in circuits])
    with qs.Batch(nq, nl) as b:
        got = b.run(angles)
    for i, c in enumerate(circuits):
        assert abs(got[i] - want[i]) <= tol(c["n"]), (c["n"], got[i], want[i])


def test_full_batch_4096_sampled(qs, oracle_mod):
    circuits = cg.hea_batch(4096, seed=2016)
    nq = [c["n"] for c in circuits]
    nl = [c["L"] for c in circuits]
    angles = qs.hea_angles(circuits)
    with qs.Batch(nq, nl) as b:
        cfg = b.autotune(angles, reps=2)
        got = b.run(angles)
    assert np.all(np.isfinite(got))
    # stratified sample: two circuits per qubit count
    picked = []
    for n in range(10, 21):
        idx = [i for i, c in enumerate(circuits) if c["n"] == n][:2]
        picked += idx
    for i in picked:
        want = oracle_energy(oracle_mod, circuits[i])
        assert abs(got[i] - want) <= tol(circuits[i]["n"]), (i, circuits[i]["n"], got[i], want)
    print("autotuned config (threads, m):", cfg)


def test_batch_rejects_bad_input(qs):
    with pytest.raises(qs.QsimError):
        qs.Batch([1, 5], [1, 1])
    with qs.Batch([4, 5], [1, 2]) as b:
        with pytest.raises(ValueError):
            b.run(np.zeros(3))
        bad = np.zeros(2 * 4 * 1 + 2 * 5 * 2)
        bad[3] = np.nan
        with pytest.raises(qs.QsimError) as e:
            b.run(bad)
        assert e.value.status == "ENONFINITE"
        with pytest.raises(qs.QsimError):
            b.set_config(256, 14)

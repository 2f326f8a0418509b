"""The allocation-free probabilities call, checked against the oracle and
the regular one.

qsim_probs_all_noalloc serves callers that cannot allocate GPU memory when
they ask for probabilities (their device memory belongs to another pool, a
fixed real-time budget, an allocation-free callback).  It must give what the
FP64 oracle and sim_probs_all give, within the tests' tolerances, on
consecutive calls that share its built-in scratch array, and it must leave
the device's free memory unchanged.  This file is named to be collected
last.
"""
import ctypes

import numpy as np
import pytest

import circuitgen as cg

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    fn = lib.qsim_probs_all_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


# 7: the one-block kernel; 10: the smallest tiled register; 16: several
# tiles per CTA; 24: more tiles than the grid holds (grid-stride loop)
@pytest.mark.parametrize("prec,tol", [("c128", 1e-12), ("c64", 1e-6)])
def test_noalloc_probs_match_oracle_and_sim_probs_all(prec, tol, oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1612_08091_gb300 as q

    fn = _noalloc(q.load())
    precision = 0 if prec == "c128" else 1
    stream = torch.cuda.current_stream()
    for n in (7, 10, 16, 24):
        psi = cg.random_state(n, seed=40 + n)
        second = [cg.op("U3", (n - 1,), (), (0.7, 1.1, -0.4)), cg.op("X", (0,), (3,))]
        with q.Simulator(n, precision=prec) as sim:
            sim.set_amplitudes(psi)
            out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
            for call in range(2):
                ref = oracle_mod.OracleSim(n, psi=psi)
                if call == 1:  # change the state between the two calls
                    sim.run(second)
                    oracle_mod.run_ops(ref, second)
                ref_p1, ref_norm = sim.probs_all()
                ptr = sim.state_ptr()
                torch.cuda.synchronize()
                free_before = torch.cuda.mem_get_info()[0]
                rc = fn(ptr, n, precision, out.data_ptr(), stream.cuda_stream)
                assert rc == 0
                torch.cuda.synchronize()
                if call == 1:  # the first call on the device may load the module
                    assert torch.cuda.mem_get_info()[0] == free_before
                got = out.cpu().numpy()
                # against the regular entry point
                assert abs(got[0] - ref_norm) <= tol
                np.testing.assert_allclose(got[1:], ref_p1, atol=tol)
                # against the FP64 oracle (complex64: the amplitudes themselves
                # are rounded to FP32, relative 2^-24 each)
                assert abs(got[0] - ref.norm2()) <= tol
                np.testing.assert_allclose(got[1:], ref.probs_all(), atol=tol)
    # sizes beyond the scratch array and bad arguments are rejected
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert fn(dummy.data_ptr(), 37, precision, dummy.data_ptr(), None) == 9  # ENOTSUP
    assert fn(None, 5, precision, dummy.data_ptr(), None) == 1  # EINVAL
    assert fn(dummy.data_ptr(), 5, 3, dummy.data_ptr(), None) == 1


def test_noalloc_probs_33_qubits_basis_state():
    """Qubits 32 and above (their partial sums take a second per-lane
    accumulator): a 33-qubit complex64 register (64 GiB) in a basis state
    with bit 32 set; every probability is exactly 0 or 1."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1612_08091_gb300 as q

    fn = _noalloc(q.load())
    n = 33
    basis = (1 << 32) | (1 << 20) | (1 << 5) | 1
    out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    with q.Simulator(n, precision="c64") as sim:
        sim.reset(basis)
        ptr = sim.state_ptr()
        assert fn(ptr, n, 1, out.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert got[0] == 1.0
    np.testing.assert_array_equal(got[1:], [(basis >> k) & 1 for k in range(n)])
    torch.cuda.empty_cache()

"""The device-side bounded wait, made to run out: a kernel polls an mbarrier
that nothing arrives on (the same helper every bulk-copy and tensor-core
wait uses), gives up after its bound, raises the error flag, and the host
reports QSIM_ETIMEOUT with the context still usable."""
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


def test_bounded_wait_times_out_and_context_survives(qs, oracle_mod):
    times = {}
    for limit in (1, 256, 4096):
        status, ms = qs.selftest_wait_timeout(limit)
        assert status == "ETIMEOUT", (limit, status)
        times[limit] = ms
    per_poll_us = 1e3 * (times[4096] - times[1]) / 4095
    print("bounded wait: %.3f us per poll; the kernels' bound of 2^18 polls gives up after about %.2f s"
          % (per_poll_us, per_poll_us * (1 << 18) / 1e6))
    assert times[4096] < 5e3  # the wait ended by its bound, not by a watchdog
    # the context still runs kernels and gives correct results
    n = 12
    ops = cg.random_u3_brickwork(n, 4, seed=3)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    with qs.Simulator(n, precision="c128") as sim:
        sim.run(ops)
        got = sim.get_amplitudes()
    assert np.max(np.abs(got - ref.psi)) <= 1e-12


def test_selftest_rejects_bad_limit(qs):
    for bad in (0, (1 << 20) + 1):
        status, _ = qs.selftest_wait_timeout(bad)
        assert status == "EINVAL"

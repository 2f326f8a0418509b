"""Handle-level behaviour of the C ABI on the GPU: library-owned against
caller-owned (torch) memory, caller streams and sim_set_stream, the raw
state pointer read as a device array without a copy, two handles used in
turn, and checkpoint / resume through get and set amplitudes."""
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


@pytest.mark.parametrize("prec,fusion", [("c128", "none"), ("c64", "greedy")])
def test_library_memory_matches_torch_memory(qs, prec, fusion):
    n = 16
    ops = cg.random_u3_brickwork(n, 6, seed=21)
    out = []
    for torch_memory in (True, False):
        with qs.Simulator(n, precision=prec, fusion=fusion, torch_memory=torch_memory) as sim:
            sim.run(ops)
            out.append(sim.get_amplitudes())
    # the same kernels on the same inputs (complex64: the norm tracking's
    # FP64 sums may round in another order)
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=0 if prec == "c128" else 1e-7)


def test_caller_streams(qs, oracle_mod):
    import torch

    n = 15
    ops = cg.random_u3_brickwork(n, 6, seed=22)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with qs.Simulator(n, precision="c128", stream=s1) as sim:
        sim.run(ops[: len(ops) // 2])
        sim.flush()
        sim.set_stream(s2)  # later work on the other stream
        sim.run(ops[len(ops) // 2:])
        sim.flush()
        s2.synchronize()
        got = sim.get_amplitudes()
    assert np.max(np.abs(got - ref.psi)) <= 1e-12


class _DeviceArray:
    """A device pointer described by __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_state_pointer_zero_copy(qs, prec):
    import torch

    n = 12
    with qs.Simulator(n, precision=prec) as sim:
        sim.run(cg.random_u3_brickwork(n, 3, seed=23))
        sim.flush()
        torch.cuda.synchronize()
        typestr = "<c16" if prec == "c128" else "<c8"
        view = torch.as_tensor(_DeviceArray(sim.state_ptr(), 1 << n, typestr), device="cuda")
        got = view.cpu().numpy().astype(np.complex128)
        want = sim.get_amplitudes()
    np.testing.assert_array_equal(got, want)


def test_two_handles_in_turn(qs, oracle_mod):
    na, nb = 13, 17
    opsa = cg.random_u3_brickwork(na, 8, seed=24)
    opsb = cg.random_u3_brickwork(nb, 8, seed=25)
    refa, refb = oracle_mod.OracleSim(na), oracle_mod.OracleSim(nb)
    oracle_mod.run_ops(refa, opsa)
    oracle_mod.run_ops(refb, opsb)
    with qs.Simulator(na, precision="c128") as a, qs.Simulator(nb, precision="c64", fusion="greedy") as b:
        step = 10
        for i in range(0, max(len(opsa), len(opsb)), step):
            a.run(opsa[i:i + step])
            b.run(opsb[i:i + step])
            if i % (3 * step) == 0:  # flushes interleaved with queued work
                a.flush()
                b.probs_all()
        ga, gb = a.get_amplitudes(), b.get_amplitudes()
    assert np.max(np.abs(ga - refa.psi)) <= 1e-12
    assert infidelity(refb.psi, gb) <= TOL64_INFID


@pytest.mark.parametrize("prec,fusion", [("c128", "none"), ("c64", "greedy")])
def test_checkpoint_and_resume(qs, prec, fusion):
    n = 18
    ops = cg.random_u3_brickwork(n, 10, seed=26)
    half = len(ops) // 2
    with qs.Simulator(n, precision=prec, fusion=fusion) as sim:
        sim.run(ops)
        straight = sim.get_amplitudes()
    with qs.Simulator(n, precision=prec, fusion=fusion) as sim:
        sim.run(ops[:half])
        ckpt = sim.get_amplitudes()
    with qs.Simulator(n, precision=prec, fusion=fusion) as sim:
        sim.set_amplitudes(ckpt)
        sim.run(ops[half:])
        resumed = sim.get_amplitudes()
    if prec == "c128":
        np.testing.assert_array_equal(resumed, straight)
    else:
        # the fused plan differs at the cut; complex64 rounding only
        assert infidelity(straight, resumed) <= TOL64_INFID

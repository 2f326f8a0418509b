"""FP64 CPU oracle for the state-vector hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in ``paper_1612_08091_gb300``
and never imports it; the only thing both sides consume is the seeded circuit
description produced by ``circuitgen``.

Layout:
  qsim_oracle.c   plain C loops over all 2^n indices (gate, probability,
                  collapse, sampling), compiled by :func:`build` with gcc.
  gates.py        the oracle's own gate matrices, written from their
                  textbook definitions.
  sim.py          :class:`OracleSim`, the register plus Pauli-sum
                  expectation done the slow way (apply the Pauli factors as
                  gates to a copy, then take the inner product).
"""
from .build import build, library_path  # noqa: F401
from .sim import OracleSim, run_ops  # noqa: F401
from . import gates  # noqa: F401

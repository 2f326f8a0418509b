"""Shared test helpers: fidelity metrics and tolerances.

Tolerances (per result, against the FP64 oracle):
  complex128 plain path: max |amplitude error| <= 1e-11, probabilities and
      expectation values within 1e-11 * max(1, sum |c_k|);
  complex64 paths: state infidelity 1 - |<a|b>|^2 / (|a|^2 |b|^2) <= 1e-5,
      probabilities within 1e-5 and expectation values within
      1e-5 * max(1, sum |c_k|).
"""
import numpy as np

TOL128_AMP = 1e-11
TOL64_INFID = 1e-5
TOL64_PROB = 1e-5


def infidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    return float(1.0 - abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def expect_tol(terms, base):
    return base * max(1.0, sum(abs(c) for c, _, _ in terms))

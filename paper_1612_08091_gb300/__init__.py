"""GB300 (sm_103a) dense state-vector simulator: CUDA kernels behind the C ABI
of include/qsim.h, with a thin ctypes binding (:mod:`.qsim`)."""
from .qsim import Simulator, Batch, QsimError, load, LIB_PATH, hea_angles, selftest_wait_timeout  # noqa: F401
from . import gates  # noqa: F401

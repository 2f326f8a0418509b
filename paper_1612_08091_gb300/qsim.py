"""Python binding of libqsim: the C ABI of include/qsim.h, one method per call.

Argument marshalling only -- every step on amplitudes runs in the library's
CUDA kernels.  Device memory for the state and the scratch workspace is
allocated through PyTorch's caching allocator and handed to ``sim_create``;
work runs on the current PyTorch CUDA stream unless another is given.  There
is no CPU fallback: without the built library or a GPU, construction fails.
"""
import ctypes
import os

import numpy as np

from . import gates as _gates

C128, C64 = 0, 1
FUSE_NONE, FUSE_GREEDY, FUSE_MLP = 0, 1, 2
_PREC = {"c128": C128, "complex128": C128, "c64": C64, "complex64": C64, C128: C128, C64: C64}
_FUSE = {"none": FUSE_NONE, "greedy": FUSE_GREEDY, "mlp": FUSE_MLP, FUSE_NONE: FUSE_NONE,
         FUSE_GREEDY: FUSE_GREEDY, FUSE_MLP: FUSE_MLP}

STATUS = {0: "OK", 1: "EINVAL", 2: "ERANGE", 3: "EDUP", 4: "ENOMEM", 5: "EZEROPROB", 6: "ENONFINITE",
          7: "ECUDA", 8: "ETIMEOUT", 9: "ENOTSUP"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")
_lib = None


class QsimError(RuntimeError):
    def __init__(self, code, call, msg):
        super().__init__("%s failed: %s (%s)" % (call, STATUS.get(code, code), msg))
        self.code = code
        self.status = STATUS.get(code, str(code))


class Opts(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p), ("state_bytes", ctypes.c_size_t),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("fusion", ctypes.c_int), ("kmax", ctypes.c_int),
                ("device", ctypes.c_int), ("tc_terms", ctypes.c_int), ("no_tensor_cores", ctypes.c_int),
                ("no_norm_tracking", ctypes.c_int), ("c128_double_float", ctypes.c_int),
                ("no_permutation_blocks", ctypes.c_int),
                ("no_product_passes", ctypes.c_int)]


class Pauli(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("gates", ctypes.c_uint64), ("passes", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("amp_updates", ctypes.c_double), ("alg_bytes", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double)]


def load():
    """Load libqsim.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from .build import build
        build()
    lib = ctypes.CDLL(LIB_PATH)
    P, I, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "sim_workspace_bytes": [I, I, ctypes.POINTER(ctypes.c_size_t)],
        "sim_create": [I, I, ctypes.POINTER(Opts), ctypes.POINTER(P)],
        "sim_destroy": [P],
        "sim_reset": [P, U64],
        "sim_apply": [P, DP, IP, I, IP, I],
        "sim_flush": [P],
        "sim_prob": [P, I, DP],
        "sim_probs_all": [P, DP, DP],
        "sim_measure": [P, I, D, IP, DP],
        "sim_collapse": [P, IP, I, IP, DP],
        "sim_measure_all": [P, D, ctypes.POINTER(U64)],
        "sim_expect": [P, ctypes.POINTER(Pauli), I, DP],
        "sim_get_amplitudes": [P, U64, U64, DP],
        "sim_set_amplitudes": [P, U64, U64, DP],
        "sim_state_ptr": [P, ctypes.POINTER(P)],
        "sim_set_stream": [P, P],
        "sim_set_fusion": [P, I, I],
        "sim_get_stats": [P, ctypes.POINTER(Stats)],
        "sim_reset_stats": [P],
        "sim_set_profiling": [P, I],
        "sim_apply_permutation": [P, ctypes.POINTER(U64), IP, I, IP, I],
        "sim_batch_workspace_bytes": [I, IP, IP, ctypes.POINTER(ctypes.c_size_t)],
        "sim_batch_create": [I, IP, IP, D, P, P, ctypes.c_size_t, ctypes.POINTER(P)],
        "sim_batch_run": [P, DP, DP],
        "sim_batch_autotune": [P, DP, I, IP, IP],
        "sim_batch_set_config": [P, I, I],
        "sim_batch_destroy": [P],
        "sim_get_kernel_times": [P, ctypes.POINTER(KernelTime), I, IP],
        "sim_swap_halves": [P, P, I],
        "sim_project": [P, IP, I, IP, D, D],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.sim_batch_last_error.argtypes = [P]
    lib.sim_batch_last_error.restype = ctypes.c_char_p
    lib.sim_last_error.argtypes = [P]
    lib.sim_last_error.restype = ctypes.c_char_p
    lib.qsim_build_info.argtypes = []
    lib.qsim_build_info.restype = ctypes.c_char_p
    lib.qsim_selftest_wait_timeout.argtypes = [ctypes.c_uint, P, DP]
    lib.qsim_selftest_wait_timeout.restype = ctypes.c_int
    _lib = lib
    return lib


def selftest_wait_timeout(limit, stream=None):
    """Run the device's bounded mbarrier wait on a barrier nothing arrives
    on (qsim_selftest_wait_timeout); returns (status name, kernel ms)."""
    lib = load()
    ms = ctypes.c_double()
    code = lib.qsim_selftest_wait_timeout(int(limit), ctypes.c_void_p(stream), ctypes.byref(ms))
    return STATUS.get(code, str(code)), ms.value


def _ints(seq):
    seq = [int(v) for v in seq]
    return (ctypes.c_int * max(1, len(seq)))(*seq), len(seq)


class Simulator:
    """An n-qubit register on the GPU behind the libqsim C ABI."""

    def __init__(self, n, precision="c128", fusion="none", kmax=6, device=None, stream=None, torch_memory=True,
                 tc_terms=3, tensor_cores=True, norm_tracking=True, c128_df=False, perm_blocks=True,
                 product_passes=True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libqsim needs a CUDA GPU; none is visible")
        self.lib = load()
        self.n = int(n)
        self.precision = _PREC[precision]
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        amp = 16 if self.precision == C128 else 8
        opts = Opts()
        opts.fusion = _FUSE[fusion]
        opts.kmax = int(kmax)
        opts.device = dev
        opts.tc_terms = int(tc_terms)
        opts.no_tensor_cores = 0 if tensor_cores else 1
        opts.no_norm_tracking = 0 if norm_tracking else 1
        opts.c128_double_float = 1 if c128_df else 0
        opts.no_permutation_blocks = 0 if perm_blocks else 1
        opts.no_product_passes = 0 if product_passes else 1
        self._keep = []
        if torch_memory:
            ws = ctypes.c_size_t()
            self._check(self.lib.sim_workspace_bytes(self.n, self.precision, ctypes.byref(ws)), "sim_workspace_bytes")
            state = torch.empty(amp << self.n, dtype=torch.uint8, device=self.device)
            work = torch.empty(ws.value, dtype=torch.uint8, device=self.device)
            self._keep += [state, work]
            opts.state, opts.state_bytes = state.data_ptr(), state.numel()
            opts.workspace, opts.workspace_bytes = work.data_ptr(), work.numel()
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        opts.stream = s.cuda_stream if hasattr(s, "cuda_stream") else int(s)
        self._stream = s
        h = ctypes.c_void_p()
        rc = self.lib.sim_create(self.n, self.precision, ctypes.byref(opts), ctypes.byref(h))
        if rc:
            raise QsimError(rc, "sim_create", "n=%d" % self.n)
        self.h = h

    # -- plumbing --------------------------------------------------------------
    def _check(self, rc, call):
        if rc:
            msg = self.lib.sim_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise QsimError(rc, call, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_destroy(self.h)
            self.h = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the C ABI -------------------------------------------------------------
    def reset(self, basis=0):
        self._check(self.lib.sim_reset(self.h, int(basis)), "sim_reset")

    def apply(self, matrix, targets, controls=()):
        m = np.ascontiguousarray(matrix, dtype=np.complex128)
        buf = m.view(np.float64)
        t, nt = _ints(targets)
        c, nc = _ints(controls)
        self._check(self.lib.sim_apply(self.h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), t, nt,
                                       c if nc else None, nc), "sim_apply")

    def apply_op(self, op):
        self.apply(_gates.gate_matrix(op.kind, op.params), op.targets, op.controls)

    def run(self, ops):
        for op in ops:
            self.apply_op(op)

    def flush(self):
        self._check(self.lib.sim_flush(self.h), "sim_flush")

    def apply_permutation(self, perm, qubits, controls=()):
        """Emulate a classical bijection on the register `qubits` (bit j of
        the register value is qubits[j]): x -> perm[x] where all controls
        are |1> (sim_apply_permutation)."""
        p = np.ascontiguousarray(perm, dtype=np.uint64)
        q, m = _ints(qubits)
        c, nc = _ints(controls)
        self._check(self.lib.sim_apply_permutation(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), q, m,
                                                   c if nc else None, nc), "sim_apply_permutation")

    def prob(self, qubit):
        out = ctypes.c_double()
        self._check(self.lib.sim_prob(self.h, int(qubit), ctypes.byref(out)), "sim_prob")
        return out.value

    def probs_all(self):
        p = np.zeros(self.n)
        nrm = ctypes.c_double()
        self._check(self.lib.sim_probs_all(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.byref(nrm)), "sim_probs_all")
        return p, nrm.value

    def measure(self, qubit, u):
        out = ctypes.c_int()
        p = ctypes.c_double()
        self._check(self.lib.sim_measure(self.h, int(qubit), float(u), ctypes.byref(out), ctypes.byref(p)),
                    "sim_measure")
        return out.value, p.value

    def collapse(self, qubits, bits):
        q, m = _ints(qubits)
        b, _ = _ints(bits)
        p = ctypes.c_double()
        self._check(self.lib.sim_collapse(self.h, q, m, b, ctypes.byref(p)), "sim_collapse")
        return p.value

    def project(self, qubits, bits, scale, kept_norm2=-1.0):
        """Keep the amplitudes with qubits[j] == bits[j], multiplied by
        `scale`; zero the rest (sim_project).  kept_norm2: their squared
        norm before scaling if known (else negative)."""
        q, m = _ints(qubits)
        b, _ = _ints(bits)
        self._check(self.lib.sim_project(self.h, q if m else None, m, b if m else None, float(scale),
                                         float(kept_norm2)), "sim_project")

    def swap_halves(self, other, qubit):
        """Exchange amplitude i + 2^qubit of this handle with amplitude i of
        `other` for every i with bit `qubit` clear (sim_swap_halves)."""
        self._check(self.lib.sim_swap_halves(self.h, other.h, int(qubit)), "sim_swap_halves")

    def measure_all(self, u):
        out = ctypes.c_uint64()
        self._check(self.lib.sim_measure_all(self.h, float(u), ctypes.byref(out)), "sim_measure_all")
        return int(out.value)

    def expect(self, terms):
        arr = (Pauli * max(1, len(terms)))()
        for k, (c, x, z) in enumerate(terms):
            arr[k] = Pauli(float(c), int(x), int(z))
        out = ctypes.c_double()
        self._check(self.lib.sim_expect(self.h, arr, len(terms), ctypes.byref(out)), "sim_expect")
        return out.value

    def get_amplitudes(self, offset=0, count=None):
        if count is None:
            count = (1 << self.n) - offset
        out = np.empty(count, dtype=np.complex128)
        self._check(self.lib.sim_get_amplitudes(self.h, int(offset), int(count),
                                                out.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "sim_get_amplitudes")
        return out

    def set_amplitudes(self, values, offset=0):
        v = np.ascontiguousarray(values, dtype=np.complex128)
        self._check(self.lib.sim_set_amplitudes(self.h, int(offset), len(v),
                                                v.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "sim_set_amplitudes")

    def state_ptr(self):
        p = ctypes.c_void_p()
        self._check(self.lib.sim_state_ptr(self.h, ctypes.byref(p)), "sim_state_ptr")
        return p.value

    def set_stream(self, stream):
        self._stream = stream
        self._check(self.lib.sim_set_stream(self.h, stream.cuda_stream if hasattr(stream, "cuda_stream")
                                            else int(stream)), "sim_set_stream")

    def set_fusion(self, mode, kmax=6):
        self._check(self.lib.sim_set_fusion(self.h, _FUSE[mode], int(kmax)), "sim_set_fusion")

    def stats(self):
        st = Stats()
        self._check(self.lib.sim_get_stats(self.h, ctypes.byref(st)), "sim_get_stats")
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def reset_stats(self):
        self._check(self.lib.sim_reset_stats(self.h), "sim_reset_stats")

    def set_profiling(self, on=True):
        """on: False/0 off, True/1 per-class times, 2 also per-launch records."""
        mode = int(on) if not isinstance(on, bool) else (1 if on else 0)
        self._check(self.lib.sim_set_profiling(self.h, mode), "sim_set_profiling")

    def kernel_times(self):
        rows = (KernelTime * 16)()
        nr = ctypes.c_int()
        self._check(self.lib.sim_get_kernel_times(self.h, rows, 16, ctypes.byref(nr)), "sim_get_kernel_times")
        return {rows[i].name.decode(): {"launches": rows[i].launches, "total_ms": rows[i].total_ms,
                                        "alg_bytes": rows[i].alg_bytes} for i in range(min(nr.value, 16))}


class Batch:
    """A batch of hardware-efficient-ansatz circuits evaluated in one
    persistent launch (sim_batch_* in the C ABI)."""

    def __init__(self, nqubits, layers, h=0.7, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libqsim needs a CUDA GPU; none is visible")
        self.lib = load()
        self.count = len(nqubits)
        self.nq = np.ascontiguousarray(nqubits, dtype=np.int32)
        self.nl = np.ascontiguousarray(layers, dtype=np.int32)
        self.nangles = int(np.sum(2 * self.nq.astype(np.int64) * self.nl))
        ip = ctypes.POINTER(ctypes.c_int)
        nbytes = ctypes.c_size_t()
        rc = self.lib.sim_batch_workspace_bytes(self.count, self.nq.ctypes.data_as(ip), self.nl.ctypes.data_as(ip),
                                                ctypes.byref(nbytes))
        if rc:
            raise QsimError(rc, "sim_batch_workspace_bytes", "")
        self._ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        self._stream = stream if stream is not None else torch.cuda.Stream()
        h_ = ctypes.c_void_p()
        rc = self.lib.sim_batch_create(self.count, self.nq.ctypes.data_as(ip), self.nl.ctypes.data_as(ip), float(h),
                                       self._stream.cuda_stream, self._ws.data_ptr(), self._ws.numel(),
                                       ctypes.byref(h_))
        if rc:
            raise QsimError(rc, "sim_batch_create", "")
        self.h = h_

    def _check(self, rc, call):
        if rc:
            raise QsimError(rc, call, self.lib.sim_batch_last_error(self.h).decode())

    def _angles(self, angles):
        a = np.ascontiguousarray(angles, dtype=np.float64)
        if a.size != self.nangles:
            raise ValueError("expected %d angles, got %d" % (self.nangles, a.size))
        return a

    def run(self, angles):
        a = self._angles(angles)
        out = np.empty(self.count, dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.sim_batch_run(self.h, a.ctypes.data_as(dp), out.ctypes.data_as(dp)), "sim_batch_run")
        return out

    def autotune(self, angles, reps=3):
        a = self._angles(angles)
        t, m = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.sim_batch_autotune(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(reps),
                                                ctypes.byref(t), ctypes.byref(m)), "sim_batch_autotune")
        return t.value, m.value

    def set_config(self, threads, m):
        self._check(self.lib.sim_batch_set_config(self.h, int(threads), int(m)), "sim_batch_set_config")

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def hea_angles(circuits):
    """Flatten circuitgen.hea_batch entries into the sim_batch_run layout."""
    parts = []
    for c in circuits:
        for l in range(c["L"]):
            parts.append(np.asarray(c["ry"][l], dtype=np.float64))
            parts.append(np.asarray(c["rz"][l], dtype=np.float64))
    return np.concatenate(parts) if parts else np.zeros(0)


def _bind_learned(lib):
    if getattr(lib, "_learned_bound", False):
        return lib
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    FP, IP = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)
    sig = {
        "sim_get_item_times": [P, FP, FP, I, IP],
        "sim_set_cost_model": [P, FP, I, I],
        "sim_plan_stats": [P, ctypes.POINTER(D)],
        "sim_mlp_create": [I, ctypes.c_ulonglong, P, ctypes.POINTER(P)],
        "sim_mlp_destroy": [P],
        "sim_mlp_get_params": [P, FP, I],
        "sim_mlp_set_params": [P, FP, I],
        "sim_mlp_forward": [P, FP, I, FP],
        "sim_mlp_gradient": [P, FP, FP, I, FP, FP],
        "sim_mlp_train": [P, FP, FP, I, I, I, ctypes.c_float, FP],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.sim_mlp_param_count.argtypes = [I]
    lib.sim_mlp_param_count.restype = I
    lib._learned_bound = True
    return lib


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


NFEATURES = 16


def _sim_item_times(self):
    lib = _bind_learned(self.lib)
    n = ctypes.c_int()
    self._check(lib.sim_get_item_times(self.h, None, None, 0, ctypes.byref(n)), "sim_get_item_times")
    feats = np.zeros((max(1, n.value), NFEATURES), dtype=np.float32)
    ms = np.zeros(max(1, n.value), dtype=np.float32)
    self._check(lib.sim_get_item_times(self.h, _fp(feats), _fp(ms), n.value, ctypes.byref(n)), "sim_get_item_times")
    return feats[:n.value], ms[:n.value]


def _sim_set_cost_model(self, params, hidden):
    lib = _bind_learned(self.lib)
    if params is None:
        self._check(lib.sim_set_cost_model(self.h, None, 0, 0), "sim_set_cost_model")
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    self._check(lib.sim_set_cost_model(self.h, _fp(p), p.size, int(hidden)), "sim_set_cost_model")


def _sim_plan_predicted_ms(self):
    lib = _bind_learned(self.lib)
    v = ctypes.c_double()
    self._check(lib.sim_plan_stats(self.h, ctypes.byref(v)), "sim_plan_stats")
    return v.value


Simulator.item_times = _sim_item_times
Simulator.set_cost_model = _sim_set_cost_model
Simulator.plan_predicted_ms = _sim_plan_predicted_ms


class MLP:
    """The cost model's network on the GPU (sim_mlp_* in the C ABI):
    16 -> hidden -> hidden -> 1, ReLU, trained with Adam on squared error."""

    def __init__(self, hidden=32, seed=1):
        self.lib = _bind_learned(load())
        self.hidden = int(hidden)
        self.nparams = self.lib.sim_mlp_param_count(self.hidden)
        h = ctypes.c_void_p()
        rc = self.lib.sim_mlp_create(self.hidden, int(seed), None, ctypes.byref(h))
        if rc:
            raise QsimError(rc, "sim_mlp_create", "")
        self.h = h

    def _check(self, rc, call):
        if rc:
            raise QsimError(rc, call, "")

    @property
    def params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        self._check(self.lib.sim_mlp_get_params(self.h, _fp(p), p.size), "sim_mlp_get_params")
        return p

    @params.setter
    def params(self, value):
        p = np.ascontiguousarray(value, dtype=np.float32)
        self._check(self.lib.sim_mlp_set_params(self.h, _fp(p), p.size), "sim_mlp_set_params")

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(X.shape[0], dtype=np.float32)
        self._check(self.lib.sim_mlp_forward(self.h, _fp(X), X.shape[0], _fp(y)), "sim_mlp_forward")
        return y

    def gradient(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(self.lib.sim_mlp_gradient(self.h, _fp(X), _fp(T), X.shape[0], _fp(g), ctypes.byref(loss)),
                    "sim_mlp_gradient")
        return g, loss.value

    def train(self, X, T, epochs=200, batch=256, lr=3e-3):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(self.lib.sim_mlp_train(self.h, _fp(X), _fp(T), X.shape[0], int(epochs), int(batch),
                                           float(lr), ctypes.byref(loss)), "sim_mlp_train")
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

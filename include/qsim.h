/*
 * qsim.h -- C ABI of libqsim, a GB300 (sm_103a) dense state-vector simulator.
 *
 * The library applies quantum gates to a dense vector of 2^n complex
 * amplitudes held in GPU memory, the operation the ProjectQ paper's
 * high-performance simulator performs one gate at a time (arXiv:1612.08091,
 * Sec. 4.3.2 "Simulation of quantum circuits").  Gates are queued lazily and
 * executed on flush, optionally fused into dense k-qubit blocks (the "lazy
 * evaluation of gates" of Sec. 4.3.2, Fig. 7 caption).  Reads -- probability,
 * measurement with collapse, Pauli-sum expectation, amplitude copies -- flush
 * first, as reading a measurement result does in the paper (Sec. 4, listing
 * 1: eng.flush() before int(qubit)).
 *
 * Conventions (the paper leaves them open; they hold for every call):
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - a gate on targets t[0..k-1] is a 2^k x 2^k matrix whose row/column
 *     index r has bit j equal to the value of qubit t[j];
 *   - host matrices are row-major complex double, (re, im) interleaved:
 *     2 * 4^k doubles;
 *   - controls fire on |1> (Sec. 4.1.3, Control meta-instruction);
 *   - device amplitudes are interleaved (re, im), complex128 (16 B) or
 *     complex64 (8 B), contiguous, 2^n of them, 256-byte aligned.
 *
 * Errors: every call returns QSIM_OK (0) or a positive status code; nothing
 * throws across the ABI.  sim_last_error() gives a one-line message for the
 * last failed call on that handle.  A call that fails validation changes
 * neither the queue nor the state.  A CUDA failure (QSIM_ECUDA) leaves the
 * state undefined.
 *
 * Ownership: the caller owns every host buffer passed in and out; matrices
 * are copied during sim_apply.  Device buffers are either passed in by the
 * caller through qsim_opts (then the caller keeps ownership and must keep
 * them alive until sim_destroy) or allocated by the library and freed in
 * sim_destroy.
 *
 * Threads and streams: a handle is used by one host thread at a time.  All
 * device work of a handle runs in order on its stream (qsim_opts.stream or
 * sim_set_stream); calls that return a host value synchronise that stream.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsim qsim;

enum qsim_status {
    QSIM_OK = 0,
    QSIM_EINVAL = 1,      /* bad argument (size, pointer, matrix shape, u outside [0,1)) */
    QSIM_ERANGE = 2,      /* qubit index outside [0, n) */
    QSIM_EDUP = 3,        /* a qubit named twice among targets and controls */
    QSIM_ENOMEM = 4,      /* device or host allocation failed, or buffer too small */
    QSIM_EZEROPROB = 5,   /* projection onto an outcome of probability 0 */
    QSIM_ENONFINITE = 6,  /* matrix entry or amplitude is NaN or infinite */
    QSIM_ECUDA = 7,       /* a CUDA call failed; see sim_last_error */
    QSIM_ETIMEOUT = 8,    /* a bounded device wait gave up */
    QSIM_ENOTSUP = 9      /* combination not supported by the library */
};

enum qsim_precision {
    QSIM_C128 = 0, /* complex128 amplitudes, FP64 arithmetic */
    QSIM_C64 = 1   /* complex64 amplitudes; fused blocks on tensor cores */
};

enum qsim_fusion {
    QSIM_FUSE_NONE = 0,   /* one launch per gate ("plain") */
    QSIM_FUSE_GREEDY = 1, /* greedy grouping into blocks of <= kmax qubits */
    QSIM_FUSE_MLP = 2     /* block boundaries chosen by the learned cost model */
};

/* Creation options.  Zero-initialise and set what you need; a NULL opts
 * pointer means all defaults. */
typedef struct qsim_opts {
    void *state;            /* caller-owned device buffer for the amplitudes, or NULL */
    size_t state_bytes;     /* its size; must be >= 2^n * (16 or 8) */
    void *workspace;        /* caller-owned device scratch, or NULL */
    size_t workspace_bytes; /* its size; must be >= sim_workspace_bytes() */
    void *stream;           /* cudaStream_t to run on; NULL = legacy default stream */
    int fusion;             /* enum qsim_fusion; default QSIM_FUSE_NONE */
    int kmax;               /* largest fused block, 1..6; 0 = default 6.  6-qubit blocks run
                               only on the complex64 tensor-core path with n >= 13; elsewhere
                               kmax 6 plans blocks of at most 5 qubits */
    int device;             /* CUDA device ordinal; the current device is used if < 0 */
    int tc_terms;           /* complex64 tensor-core blocks: 3 = BF16x3 (default, 0 means 3),
                               5 = five split products (gate split in three parts) */
    int no_tensor_cores;    /* non-zero: run complex64 blocks on the CUDA cores */
    int no_norm_tracking;   /* non-zero: tensor-core block passes do not scale their
                               outputs back to the norm the state had after the last
                               reset, measurement or host write */
    int c128_double_float;  /* non-zero: complex128 gates (one-qubit dense, diagonal and
                               phase gates, multi-target dense gates) and fused blocks
                               (dense and diagonal) compute in FP32 pairs (about 2^-45
                               relative error per product) instead of FP64 arithmetic */
    int no_permutation_blocks; /* non-zero: the greedy and learned planners form no
                               permutation blocks (runs of X / CNOT / Toffoli / SWAP
                               executed as one emulated-permutation pass) */
    int no_product_passes;  /* non-zero: the greedy planner (complex64, n >= 12) forms no
                               product passes (a layer of one-qubit gates on more than
                               kmax qubits between wider gates, applied 12 qubits per
                               pass) */
} qsim_opts;

/* A Pauli-sum term c * P.  Qubit q of P is X if bit q is set in xmask only,
 * Z if in zmask only, Y if in both, identity otherwise. */
typedef struct qsim_pauli {
    double coeff;
    uint64_t xmask;
    uint64_t zmask;
} qsim_pauli;

/* Counters since creation (or the last sim_reset_stats). */
typedef struct qsim_stats {
    uint64_t gates;          /* gates accepted by sim_apply */
    uint64_t passes;         /* full- or partial-vector kernel passes for gates */
    uint64_t launches;       /* kernel launches of any kind */
    double amp_updates;      /* sum over gates of 2^(n - #controls) */
    double alg_bytes;        /* algorithmic HBM bytes of the gate passes */
} qsim_stats;

/* Scratch bytes a handle of n qubits needs (whatever the precision).  Not in
 * the paper: its simulator allocates host memory itself; here a caller may
 * hand device memory in through qsim_opts. */
int sim_workspace_bytes(int n, int precision, size_t *bytes);

/* Create an n-qubit register (1 <= n <= 36) in |0...0>: the register that
 * allocate_qureg(n) hands out (Sec. 4.1.1), its qubits starting in |0> as in
 * the first example of Sec. 4.  On success *out receives the handle.
 * QSIM_ENOMEM if the state does not fit. */
int sim_create(int n, int precision, const qsim_opts *opts, qsim **out);

/* Destroy a handle; frees what the library allocated (the deallocation of
 * a register, Sec. 4.1.1).  NULL is accepted. */
int sim_destroy(qsim *s);

/* Drop the queue and set the register to the basis state |basis>: a fresh
 * register (Sec. 4.1.1) prepared in a basis state, as the reset of a measured
 * qubit before its reuse does in Shor's example (Appendix A.3). */
int sim_reset(qsim *s, uint64_t basis);

/* Queue U (2^t x 2^t, see conventions) on targets[0..t-1], conditioned on
 * controls[0..c-1] all being |1>: the `Gate | qubits` statement of Sec. 4 on
 * a tuple of qubits (Sec. 4.1.2), inside a Control(eng, controls) section
 * (Sec. 4.1.3); executed lazily (Sec. 4.3.2, Fig. 7 caption).
 * 1 <= t <= 5, 0 <= c < n.  Validated now (range, duplicates, finite
 * entries), executed at the next flush.  U may be non-unitary; the
 * complex64 norm control then starts afresh after it. */
int sim_apply(qsim *s, const double *matrix, const int *targets, int t, const int *controls, int c);

/* Execute every queued gate: eng.flush() of Sec. 4, listing 1. */
int sim_flush(qsim *s);

/* Emulation of a classical reversible function on a register (Sec. 4.3.3,
 * BasicMathGate: e.g. AddConstant(c), x -> x + c mod 2^m; the modular
 * multiplication of Appendix A.3).  The register is qubits[0..m-1] (bit j of
 * its value is qubits[j]), 1 <= m <= 12; perm[x] = f(x) for x < 2^m must be
 * a bijection (QSIM_EINVAL otherwise).  Where all controls are |1>, the
 * amplitude of register value x moves to register value f(x).  Flushes the
 * queue, then runs at once (one pass over the touched groups; fixed points
 * of f are not touched when the register and controls lie above the lowest
 * 4 KB of amplitudes and f's cycles give at least one task per SM). */
int sim_apply_permutation(qsim *s, const uint64_t *perm, const int *qubits, int m, const int *controls, int c);

/* P(qubit = 1) = sum of |psi_i|^2 over indices with bit q set, accumulated
 * in FP64 (Sec. 4, measurement in the computational basis). */
int sim_prob(qsim *s, int qubit, double *p1);

/* p1[q] = P(qubit q = 1) for all q in one pass; p1 holds n doubles. *norm2
 * (may be NULL) receives sum_i |psi_i|^2.  The per-qubit marginals of the
 * outcome distribution of Measure | qureg (Sec. 4.3.1, Fig. 6). */
int sim_probs_all(qsim *s, double *p1, double *norm2);

/* Measure one qubit with the caller's uniform draw u in [0,1): the outcome
 * is 0 iff u * norm2 < P(qubit = 0); the register is projected onto the
 * outcome and renormalised by 1/sqrt(p) computed in FP64 (Sec. 4 listing 1;
 * Appendix A.1, A.3). *p_outcome may be NULL. */
int sim_measure(qsim *s, int qubit, double u, int *outcome, double *p_outcome);

/* Project onto qubits[j] == bits[j] (j < m) and renormalise: the state
 * after Measure | (psi, b1) has given those bits (Appendix A.1).  *p (may be
 * NULL) receives sum |psi_i|^2 over the projected part, the outcome's
 * probability for a normalised state.  A projection of probability 0 returns
 * QSIM_EZEROPROB and leaves the state unchanged. */
int sim_collapse(qsim *s, const int *qubits, int m, const int *bits, double *p);

/* Measure | qureg (Sec. 4.3.1): sample the whole register with draw u in
 * [0,1): the outcome is the smallest j with sum_{i<=j} |psi_i|^2 > u * norm2
 * (cumulative sums in FP64); the register collapses to |j> keeping the
 * phase of psi_j. */
int sim_measure_all(qsim *s, double u, uint64_t *outcome);

/* <psi| sum_k terms[k].coeff * P_k |psi>, accumulated in FP64.  Not in the
 * paper (its simulator exposes no observable); the Pauli-sum expectation the
 * variational workloads need.  The state is assumed normalised (no division
 * by the norm; complex64 block passes hold the norm, see sim_apply). */
int sim_expect(qsim *s, const qsim_pauli *terms, int nterms, double *out);

/* Copy amplitudes [offset, offset+count) to host memory as complex double
 * (2*count doubles, re/im interleaved), widening complex64 exactly.  The
 * state is the one the paper's simulator back-end holds (Sec. 4.3.2); the
 * paper names no call for reading it. */
int sim_get_amplitudes(qsim *s, uint64_t offset, uint64_t count, double *out);

/* Overwrite amplitudes [offset, offset+count) from host complex double
 * (rounded to nearest for complex64).  No normalisation is applied.  Not in
 * the paper: state preparation for tests and checkpoint / resume. */
int sim_set_amplitudes(qsim *s, uint64_t offset, uint64_t count, const double *in);

/* Device pointer of the amplitudes (valid until sim_destroy).  Flushes.
 * Not in the paper: zero-copy access for device-side consumers. */
int sim_state_ptr(qsim *s, void **dev_ptr);

/* ---------------------------------------------------------------------------
 * Sharded registers.  The paper's road map (Sec. 5) points to a distributed
 * simulator that splits the state over many nodes.  A register of n qubits
 * split by its top g qubits is held as 2^g handles of n - g qubits (shards);
 * gates on the local qubits run on each shard, a qubit of the shard index is
 * first exchanged with a local one, and reductions add the shards' FP64
 * partial results.  These two calls are the device steps that need more
 * than one shard or a scale decided over all of them.
 * --------------------------------------------------------------------------- */

/* The exchange step of a sharded register (Sec. 5, distributed simulation):
 * for every index i of a shard with bit `qubit` equal to 0, amplitude
 * i + 2^qubit of shard a trades places with amplitude i of shard b.  With a
 * the shard whose index bit j is 0 and b its partner with bit j set, this
 * exchanges the local qubit `qubit` with the global qubit j.  Both handles
 * must have the same n, precision and device; both queues are flushed first.
 * Runs on a's stream, ordered after b's queued work and before b's later
 * work, and waits for it: the kernel also sums |psi|^2 of what left each
 * shard (FP64), so that shards whose norms were known keep known norms for
 * the complex64 norm control.  QSIM_EINVAL for a == b or mismatched
 * handles. */
int sim_swap_halves(qsim *a, qsim *b, int qubit);

/* The projection step of a measurement (Sec. 4, listing 1; Appendix A.1)
 * with the renormalisation supplied by the caller: amplitudes whose
 * qubits[j] == bits[j] for all j < m are multiplied by `scale`, all others
 * set to 0 (m = 0: every amplitude is multiplied by scale; scale 0 clears
 * the register).  A sharded register projects each shard with the scale
 * 1/sqrt(p) of the outcome's probability p summed over all shards.
 * kept_norm2: sum |psi_i|^2 over the kept amplitudes before scaling, if the
 * caller knows it (the complex64 norm control then steers to scale^2 times
 * it), else any negative value. */
int sim_project(qsim *s, const int *qubits, int m, const int *bits, double scale, double kept_norm2);

/* Run subsequent work on another cudaStream_t (after the current stream's
 * queued work, which this call waits for).  Not in the paper. */
int sim_set_stream(qsim *s, void *stream);

/* Choose the fusion mode (enum qsim_fusion) and block width kmax (1..6, see
 * qsim_opts.kmax): how the lazily buffered gates are executed (Sec. 4.3.2,
 * Fig. 7 caption).
 * QSIM_FUSE_MLP uses the cost model loaded with sim_set_cost_model (greedy
 * fusion if none is loaded).  Flushes the queue first. */
int sim_set_fusion(qsim *s, int mode, int kmax);

/* Counters of qsim_stats; not in the paper. */
int sim_get_stats(const qsim *s, qsim_stats *out);
int sim_reset_stats(qsim *s);

/* Per-kernel-class device time (not in the paper).  When profiling is on, every gate or block
 * launch is bracketed by CUDA events on the handle's stream; the times are
 * collected (stream synchronised) by sim_get_kernel_times, which returns one
 * row per kernel class seen since profiling was switched on.  Class names:
 * "gate_dense", "gate_phase", "gate_diag", "gate_x" (plain gates),
 * "block_tc" (4- and 5-qubit blocks on the tensor cores), "block_tc6"
 * (6-qubit blocks), "block_dense" (blocks on CUDA cores), "block_diag"
 * (diagonal blocks), "permute", "permute_cycles" and "permute_cycles_bulk"
 * (sim_apply_permutation: tiled through shared memory, or along the cycles
 * of f through registers or through the bulk-copy engine), "product" (layers
 * of one-qubit gates, 12 qubits per pass). */
typedef struct qsim_kernel_time {
    char name[24];
    uint64_t launches;
    double total_ms;   /* sum of event-timed durations */
    double alg_bytes;  /* algorithmic HBM bytes of those launches */
} qsim_kernel_time;

/* Profiling (not in the paper).
 * on: 0 off, 1 per-class times, 2 per-class times and per-launch records
 * (features of the planned item and its cost) for sim_get_item_times. */
int sim_set_profiling(qsim *s, int on);
int sim_get_kernel_times(qsim *s, qsim_kernel_time *rows, int max_rows, int *nrows);

/* ---------------------------------------------------------------------------
 * Learned fusion planner (not in the paper).  With profiling mode 2 the
 * library records, for every gate or block launch, 16 features of the
 * planned item and its cost: the larger of its event-timed device duration
 * and the host time spent issuing it (block matrix, operand record,
 * staging, launch), since small registers are host-bound.  A cost model
 * trained on these records (sim_mlp_*) predicts the log of an item's cost
 * in ms, and QSIM_FUSE_MLP plans with it: the greedy plans for kmax = 2 up
 * to the handle's block width limit (kmax, at most 6 on the complex64
 * tensor-core path, else 5) and the all-plain plan, each block either fused
 * or left as plain gates, whichever is predicted cheaper; the plan with the
 * lowest predicted total is executed, its blocks launched as they are
 * formed.  Without a loaded model QSIM_FUSE_MLP falls back to greedy fusion.
 * Feature order: n/32, bytes per amplitude/16, fused, on tensor cores,
 * width/5, gates/32, plain dense, plain phase, plain diagonal, plain X,
 * controls/8, log2(fraction of amplitudes touched)/8, lowest qubit/32,
 * highest qubit/32, qubits below 5 /5, 1.
 * --------------------------------------------------------------------------- */

/* Learned planner (not in the paper).  Copy out (and clear) the per-launch records: feats holds 16 floats per
 * record, ms one float (the cost above, in ms); *nitems receives the number
 * of records available
 * (records are cleared only when all of them fit in max_items). */
int sim_get_item_times(qsim *s, float *feats, float *ms, int max_items, int *nitems);

/* Learned planner (not in the paper).  Load the cost model (parameter layout of sim_mlp_*: W1[h][16], b1[h],
 * W2[h][h], b2[h], w3[h], b3); count 0 unloads it.  Copied. */
int sim_set_cost_model(qsim *s, const float *params, int count, int hidden);

/* Predicted cost (ms) of the last plan made by the learned planner (not in
 * the paper). */
int sim_plan_stats(qsim *s, double *predicted_ms);

/* The cost model's network (not in the paper), trained on the GPU by the library's own
 * forward, backward and Adam kernels (FP32, deterministic). */
typedef struct qsim_mlp qsim_mlp;
int sim_mlp_param_count(int hidden);
int sim_mlp_create(int hidden, unsigned long long seed, void *stream, qsim_mlp **out);
int sim_mlp_destroy(qsim_mlp *m);
int sim_mlp_get_params(qsim_mlp *m, float *out, int count);
int sim_mlp_set_params(qsim_mlp *m, const float *in, int count);
/* Cost-model inference (not in the paper): Y[i] = network(X[i*16 .. i*16+15]);
 * host arrays. */
int sim_mlp_forward(qsim_mlp *m, const float *X, int n, float *Y);
/* Cost-model training (not in the paper): gradient (parameter layout) of the
 * mean squared error over n samples. */
int sim_mlp_gradient(qsim_mlp *m, const float *X, const float *T, int n, float *grads, float *loss);
/* Cost-model training (not in the paper): Adam (lr, betas 0.9/0.999) on the mean squared error for `epochs` passes
 * in minibatches of `batch`; *loss = mean squared error of the last epoch. */
int sim_mlp_train(qsim_mlp *m, const float *X, const float *T, int n, int epochs, int batch, float lr, float *loss);

/* ---------------------------------------------------------------------------
 * Batched variational sweep (not in the paper).  A batch of hardware-
 * efficient-ansatz circuits of different sizes is evaluated in two
 * persistent launches (circuits larger than shared memory, then the rest),
 * captured in one CUDA graph and replayed per call.
 * Circuit c has nqubits[c] qubits (2..24) and layers[c] layers; it starts in
 * |0...0>, each layer applies RY(theta) to every qubit, RZ(phi) to every
 * qubit, then CNOT(q -> q+1) for q = 0..n-2 in order.  The result is the
 * transverse-field Ising energy of each circuit,
 *   E = -sum_{i<n-1} <Z_i Z_{i+1}> - h sum_i <X_i>,
 * accumulated in FP64 (amplitudes complex64, gate arithmetic FP32).
 * --------------------------------------------------------------------------- */
typedef struct qsim_batch qsim_batch;

/* Batched sweep (not in the paper).  Device bytes a batch needs (angles, energies, queue, per-CTA buffers for
 * circuits that do not fit in shared memory). */
int sim_batch_workspace_bytes(int count, const int *nqubits, const int *layers, size_t *bytes);

/* Batched sweep (not in the paper).  Create a batch.  stream: cudaStream_t to run on (NULL: the batch creates
 * its own non-blocking stream; graph capture needs a non-default stream).
 * workspace: caller-owned device memory of sim_batch_workspace_bytes bytes,
 * 256-byte aligned, or NULL to let the library allocate.  Copies the size
 * arrays.  QSIM_EINVAL for sizes outside the ranges above. */
int sim_batch_create(int count, const int *nqubits, const int *layers, double h, void *stream, void *workspace,
                     size_t workspace_bytes, qsim_batch **out);

/* Batched sweep (not in the paper).  Evaluate all circuits.  angles (host): for each circuit in order, for each
 * layer, n RY angles (qubit 0..n-1) then n RZ angles; energies (host):
 * count doubles.  The first call captures the graph (angles H2D, queue and
 * error-flag reset, the two persistent kernels, energies and flag D2H);
 * later calls replay it.  QSIM_ETIMEOUT if a bounded device wait gave up
 * (energies then not written). */
int sim_batch_run(qsim_batch *b, const double *angles, double *energies);

/* Batched sweep (not in the paper).  Time every candidate launch configuration (threads per CTA 256/512/1024,
 * shared-memory threshold m = 12..14 qubits) on these angles, reps timed
 * runs each after one warm-up, keep the fastest (median) and report it. */
int sim_batch_autotune(qsim_batch *b, const double *angles, int reps, int *threads, int *m);

/* Batched sweep (not in the paper).  Set the launch configuration of the
 * small-circuit kernel by hand
 * (QSIM_EINVAL if it cannot run: 2^m must be <= 32 * threads for 256 and
 * 512 threads, <= 16 * 1024 for 1024); circuits with more than m qubits go
 * to the global-memory kernel (256 threads, two CTAs per SM, 2^12-amplitude
 * chunks). */
int sim_batch_set_config(qsim_batch *b, int threads, int m);

/* Batched sweep (not in the paper): destroy a batch; the last failure's
 * message. */
int sim_batch_destroy(qsim_batch *b);
const char *sim_batch_last_error(const qsim_batch *b);

/* All single-qubit probabilities of a caller-owned device state vector,
 * computed without allocating any device memory.  The paper has no
 * counterpart to this call; it exists for callers that cannot allocate GPU
 * memory when they need the result (another framework's pool owns the
 * device memory, a fixed real-time memory budget, a plugin callback that
 * forbids allocation).
 *   state      device pointer to 2^n amplitudes (complex128: 16-byte aligned,
 *              complex64: 8-byte aligned), read only;
 *   n          1..36; larger registers return QSIM_ENOTSUP because the
 *              built-in scratch array holds partial sums for at most 36
 *              qubits (320 KiB, fixed at build time);
 *   precision  QSIM_C128 or QSIM_C64;
 *   out        device pointer to n + 1 doubles, written asynchronously:
 *              out[0] = sum_i |psi_i|^2, out[1 + q] = P(qubit q = 1);
 *   stream     cudaStream_t to run on (NULL = legacy default stream).
 * Returns QSIM_EINVAL for a null or misaligned pointer or an unknown
 * precision, QSIM_ECUDA if a launch fails.  No cudaMalloc, cudaFree or
 * allocating library call is made.  The scratch is one array shared by all
 * calls in the process: calls whose kernels overlap on the GPU race on it.
 * The first call on each device looks up the array's device address and
 * the device's SM count; make it before any stream capture. */
int qsim_probs_all_noalloc(const void *state, int n, int precision, double *out, void *stream);

/* Self-test of the device-side bounded wait (not in the paper).  Every kernel that waits on an
 * mbarrier (bulk copies, tensor-core commits) polls it at most a fixed
 * number of times; on time-out it raises a flag that the host reports as
 * QSIM_ETIMEOUT, and the context stays usable.  This call runs that wait on
 * a barrier that nothing arrives on, with at most `limit` polls (1..2^20),
 * on `stream` (cudaStream_t, NULL = legacy default).  Returns QSIM_ETIMEOUT
 * (the expected outcome) and the kernel's event-timed duration in *ms (may
 * be NULL); QSIM_EINVAL for a limit outside the range, QSIM_ENOMEM or
 * QSIM_ECUDA if the 4-byte flag cannot be allocated or a call fails. */
int qsim_selftest_wait_timeout(unsigned int limit, void *stream, double *ms);

/* One-line description of the last failure on this handle ("" if none).
 * Not in the paper (its Python front end raises exceptions). */
const char *sim_last_error(const qsim *s);

/* Library build string: version, target architecture.  Not in the paper. */
const char *qsim_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */

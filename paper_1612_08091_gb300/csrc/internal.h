// internal.h -- host-side structures shared by the libqsim translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <functional>
#include <vector>

#include "../../include/qsim.h"

typedef std::complex<double> cd;

// How a queued gate is executed by the unfused path.
enum GateKind {
    GK_DENSE = 0,  // general 2^t x 2^t matrix
    GK_DIAG1 = 1,  // one target, diag(d0, d1)
    GK_PHASE = 2,  // diag(1, z) on one target: multiply amplitudes with all of
                   // (targets | controls) set to 1 by z
    GK_X = 3       // one target, [[0,1],[1,0]]: swap amplitude pairs
};

struct GateRec {
    int t = 0;
    int targets[5] = {0, 0, 0, 0, 0};
    std::vector<int> controls;
    uint64_t tmask = 0, cmask = 0;
    std::vector<cd> m;  // 4^t entries, row-major, index bit j = targets[j]
    int kind = GK_DENSE;
    bool diag = false;  // the matrix is diagonal (the gate only multiplies amplitudes by phases)
    bool perm = false;  // the matrix is a 0/1 permutation matrix (X, CNOT, Toffoli, SWAP ...)
    bool unitary = true;  // max |U U^dag - I| <= 1e-9 (else the gate may change the norm)
    std::vector<uint8_t> pmap;  // perm: target value c -> the row r with m[r][c] = 1
};

// One unit of device work produced by the planner.
struct PlanItem {
    bool fused = false;     // false: execute gates[gate] with the plain kernels
    bool diag_block = false;  // fused block of diagonal gates: one multiply per amplitude
    uint64_t dmask = 0;       // qubits of a diagonal block (up to kMaxDiagQubits)
    std::vector<cd> dtab;     // its 2^popc(dmask) factors, index bit j = j-th qubit of dmask
    bool perm_block = false;  // fused block of permutation gates: amplitudes only move
    uint64_t pmask = 0;       // qubits of a permutation block (up to kMaxPermQubits)
    std::vector<uint64_t> ptab;  // f over the 2^popc(pmask) register values (bit j = j-th qubit of pmask)
    bool prod_block = false;  // one-qubit gates on many qubits: a product of 2x2 matrices
    uint64_t qmask_prod = 0;  // its qubits
    std::vector<cd> pm;       // the 2x2 matrix of each of its qubits (ascending), row-major
    int gate = -1;
    int k = 0;              // fused block width
    int qubits[6] = {0, 0, 0, 0, 0, 0};  // sorted ascending; bit j of the block index
    std::vector<cd> m;      // 2^k x 2^k block matrix
    double amp_updates = 0; // credited to the original gates
    int ngates = 0;
    std::vector<int> members;  // queue indices of the gates it executes, in order
    double host_ms = 0;     // host time spent building its matrix (profiling)
};

// The learned cost model used by the planner (host inference).
constexpr int kFeatures = 16;
constexpr int kMaxHidden = 1024;  // widest cost-model layer
struct CostModel {
    int hidden = 0;
    std::vector<float> p;  // W1[H][16], b1[H], W2[H][H], b2[H], w3[H], b3
    bool loaded() const { return hidden > 0; }
    float predict(const float *x) const;  // predicted log(ms)
};

struct qsim {
    int n = 0;
    int prec = QSIM_C128;
    int device = 0;
    int sms = 1;  // streaming multiprocessors of the device (sizes the persistent grids)
    void *state = nullptr;
    bool own_state = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    cudaStream_t stream = nullptr;
    int fusion = QSIM_FUSE_NONE;
    int kmax = 5;
    std::vector<GateRec> queue;
    double *pinned = nullptr;  // small pinned host buffer for results
    qsim_stats stats{};
    std::string err;
    // tensor-core block path
    bool tc_enabled = true;
    int tc_terms = 3;
    bool norm_tracking = true;  // each block pass scales its outputs back to the norm target
    bool c128_df = false;       // complex128 gates and blocks in double-float arithmetic
    bool perm_blocks = true;    // the planners may form permutation blocks
    bool prod_passes = true;    // the greedy planner may form product passes (complex64)
    // norm control of the tensor-core block passes (tmem_block_kernel.cu):
    // norm_chain: the previous block pass's record describes the current
    // state (false after a reset, a measurement, host-set amplitudes or a
    // non-unitary gate); norm_target: the norm a new chain steers to (1 after
    // a reset or a measurement, <= 0: the first pass's input norm)
    bool norm_chain = false;
    double norm_target = 1.0;
    uint64_t tc_passes = 0;
    int tc_prev_grid = 0;
    unsigned char *stage_host = nullptr;  // pinned staging for block operands
    size_t stage_cursor = 0;
    // profiling: events around each launch, harvested on demand
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Pending { int cls; size_t ev; double bytes; long feat; float host_ms; };
    bool record_items = false;
    std::vector<float> pending_feats;  // features of pending launches (record_items)
    std::vector<float> item_feats;     // harvested: kFeatures floats per launch
    std::vector<float> item_ms;        // harvested: event-timed duration per launch
    CostModel cost;
    double last_plan_predicted_ms = 0;
    std::vector<Pending> pending;
    struct ClassTime { uint64_t launches = 0; double ms = 0, bytes = 0; };
    ClassTime class_time[16];  // indexed by KernelClass
};

enum KernelClass {
    KC_DENSE = 0, KC_PHASE, KC_DIAG, KC_X, KC_BLOCK_TC, KC_BLOCK_DENSE, KC_BLOCK_DIAG, KC_BLOCK_TC6, KC_PERMUTE,
    KC_PERMUTE_CYCLES, KC_PERMUTE_BULK, KC_PRODUCT, KC_COUNT
};
static_assert(KC_COUNT <= 16, "class_time holds 16 kernel classes");
constexpr int kMaxDiagQubits = 12;
constexpr int kMaxPermQubits = 12;

// Bytes of one amplitude.
inline size_t amp_bytes(const qsim *s) { return s->prec == QSIM_C128 ? 16 : 8; }


// Workspace layout (byte offsets) -----------------------------------------
constexpr size_t kWsPartials = 0;                       // reduction partials
constexpr size_t kWsPartialsBytes = 1u << 20;           // 1 MiB
constexpr size_t kWsResult = kWsPartials + kWsPartialsBytes;  // final values
constexpr size_t kWsResultBytes = 64u << 10;            // 64 KiB
constexpr size_t kWsChunk = kWsResult + kWsResultBytes; // measure-all chunk sums
constexpr size_t kWsChunkBytes = 64u << 10;
constexpr size_t kWsErr = kWsChunk + kWsChunkBytes;     // device error flags
constexpr size_t kWsErrBytes = 256;
constexpr size_t kWsNorm = kWsErr + kWsErrBytes;        // block-pass norm partials
constexpr size_t kWsNormBytes = 48u << 10;  // 2 slots x 2 sums x up to kMaxTcGrid CTAs, 2 records
constexpr int kMaxTcGrid = 1024;            // largest grid of a block pass
constexpr size_t kWsRing = kWsNorm + kWsNormBytes;      // block operand ring
constexpr size_t kWsRingBytes = 16u << 20;
constexpr size_t kWsTotal = kWsRing + kWsRingBytes;
constexpr int kMaxReduceBlocks = 2048;                  // largest reduction grid (partials fit in 1 MiB)
// Grid of the reduction kernels: four CTAs per SM.
inline int reduce_blocks(const qsim *s) { return 4 * s->sms < kMaxReduceBlocks ? 4 * s->sms : kMaxReduceBlocks; }
constexpr int kMaxChunks = 4096;

// Error helpers -------------------------------------------------------------
int set_err(qsim *s, int code, const std::string &msg);
int cuda_err(qsim *s, cudaError_t e, const char *where);

// Launchers (gate_kernels.cu) -----------------------------------------------
int launch_gate_plain(qsim *s, const GateRec &g);
int launch_block_dense(qsim *s, const int *qubits, int k, const cd *m);
// Emulated classical bijection on a register (perm_kernels.cu).
// *kind: which kernel ran: 0 tiled, 1 cycle walk through registers, 2 cycle
// walk through the bulk-copy engine
int launch_permutation(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask,
                       int *kind);

// A product of one-qubit gates on the qubits of qmask (complex64): mats
// holds each qubit's 2x2 matrix, ascending, row-major; one pass per 12
// qubits (product_kernel.cu).
int launch_product(qsim *s, uint64_t qmask, const cd *mats, int *npasses);
// The passes launch_product makes for the qubits of qmask.
int product_pass_count(uint64_t qmask);
// u = c [[s00, s01], [s10, s11]] with c > 0, real signs s = +-1 and s00 s11
// = -s01 s10 (products of H and X), to 1e-12 relative: the matrices a
// product pass takes (planner.cpp)
bool butterfly2(const cd *u);
// Diagonal block: psi_i *= d[bits of i on dmask] (diag_kernels.cu).
int launch_block_diag(qsim *s, uint64_t dmask, const cd *d);
int launch_set_basis(qsim *s, uint64_t basis);

// Copy a block operand record into the device ring (via pinned staging) on
// the handle's stream; *dev receives its device address (api.cpp).
int stage_operand(qsim *s, const void *data, size_t bytes, unsigned char **dev);
// Read and clear the device error flags (synchronises the stream).
int check_device_errors(qsim *s);

// Fused 4- or 5-qubit tensor-core block (tmem_block_kernel.cu; a 4-qubit
// block is embedded in a 5-qubit one).  Returns QSIM_ENOTSUP when the
// block cannot run on the tensor-core kernel (caller falls back).
int launch_block_tc(qsim *s, const int *qubits, int k, const cd *m);
// 5- or 6-qubit block with the state operand in tensor memory (complex64,
// tensor cores, n >= k + 7); QSIM_ENOTSUP otherwise
int launch_block_tmem(qsim *s, const int *qubits, int k, const cd *m);

// Reductions and measurement (reduce_kernels.cu) ----------------------------
int run_probs_all(qsim *s, double *p1, double *norm2);
int run_masked_sum(qsim *s, uint64_t mask, uint64_t value, double *out);
int run_split_sum(qsim *s, int q, double *s0, double *s1);
int run_collapse_mask(qsim *s, uint64_t mask, uint64_t value, double scale);
int run_expect(qsim *s, const qsim_pauli *terms, int nterms, double *out);
int run_measure_all(qsim *s, double u, uint64_t *outcome);

// Planner (planner.cpp) -------------------------------------------------------
void plan_none(const std::vector<GateRec> &q, int n, std::vector<PlanItem> &out);
// diag_k: widest diagonal block (0 disables diagonal blocks); matrices:
// build each fused block's matrix or diagonal table (false: members and
// qubits only, for comparing plans); perm_min: narrowest permutation block
// worth a pass of its own (0 disables permutation blocks; see perm_min_width);
// prod_min: fewest qubits of a product pass (0 disables them): a run of
// uncontrolled one-qubit gates on at least prod_min qubits, each of whose
// wires continues with a gate on more than kmax qubits (or ends) and has a
// butterfly2 matrix (wires whose product is the identity drop out), becomes
// one product item; tie: how the dense grower chooses among ready gates
// adding the same number of new qubits (0: the earliest; 1: the one sharing
// the most qubits with the block, then the earliest)
void plan_greedy(const std::vector<GateRec> &q, int n, int kmax, std::vector<PlanItem> &out,
                 int diag_k = kMaxDiagQubits, bool matrices = true, int perm_min = 0, int prod_min = 0,
                 int tie = 0);
// The same plan handed to emit item by item as it is formed (so execution
// overlaps planning); a non-zero return of emit stops planning and is returned.
int plan_greedy_each(const std::vector<GateRec> &q, int n, int kmax, const std::function<int(PlanItem &)> &emit,
                     int diag_k = kMaxDiagQubits, bool matrices = true, int perm_min = 0, int prod_min = 0,
                     int tie = 0);
// The narrowest permutation block the executor runs as its own pass:
// complex128 dense blocks are bound by arithmetic, so any permutation block
// of two or more gates is cheaper; complex64 dense blocks are HBM-bound like
// a permutation pass, so only a permutation block wider than any dense block
// (more than kmax qubits) saves passes.
int perm_min_width(int prec, int kmax);
// The permutation matrix of a gate as a map of its target values (perm and
// pmap of GateRec); false if the matrix is not a 0/1 permutation.
bool perm_map(const GateRec &g, std::vector<uint8_t> &pmap);
// Fill it.m, the product of the member gates embedded in it.qubits (a dense
// block), or it.dtab (a diagonal block).
void block_matrix(const std::vector<GateRec> &q, PlanItem &it);
// Features of one plan item (kFeatures floats).
// df: complex128 launches use double-float arithmetic (feature 3 = 0.5)
void item_features(const PlanItem &it, const std::vector<GateRec> &q, int n, int prec, bool tc_enabled, bool df,
                   float *f);
// Learned planner: the greedy plans for kmax = 2..kmax_limit (without block
// matrices), each block fused or left as plain gates, whichever the cost
// model predicts cheaper, against all gates plain (kmax 1); the plan with the
// lowest predicted total wins.  The choice is its kmax and, for each item of
// plan_greedy(kmax) in order, whether to run it fused (1) or as its member
// gates (0); plan_greedy_each regenerates the same items for execution.
struct MlpChoice {
    int kmax = 1;
    std::vector<char> fuse;
    double predicted_ms = 0;
};
void plan_mlp(const std::vector<GateRec> &q, int n, int prec, bool tc_enabled, bool df, bool perm_blocks,
              int kmax_limit, const CostModel &cm,
              MlpChoice &choice);
// Gate gi as a plan item of its own.
PlanItem single_item(const std::vector<GateRec> &q, int n, int gi);

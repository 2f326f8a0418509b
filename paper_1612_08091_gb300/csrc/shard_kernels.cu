// shard_kernels.cu -- the exchange step of a register split into shards.
//
// The paper's road map (Sec. 5) points to a distributed simulator that
// splits the state vector over many nodes (45 qubits).  With the register
// split by its top g qubits into 2^g shards of 2^(n-g) amplitudes, every gate
// whose targets are local qubits runs on each shard independently; a gate on
// a qubit held in the shard index ("global" qubit) first needs that qubit
// exchanged with a local one.  Exchanging global position G (shard-index bit
// j) with local position l moves every amplitude whose bits l and G differ:
// for shards s (bit j = 0) and s' = s | 2^j, amplitude i | 2^l of s trades
// places with amplitude i of s' (i with bit l = 0).  sim_swap_halves runs that
// exchange between two shards held on one device; sim_project is the
// projection step of a measurement with the renormalisation decided over all
// shards.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kSwapThreads = 256;
constexpr int kSwapPer = 4;  // pairs per thread per round: their loads go out together

// For g < npairs: i = g with a zero inserted at bit q; a[i | 2^q] <-> b[i].
template <typename Amp>
__global__ void __launch_bounds__(kSwapThreads) k_swap_halves(Amp *__restrict__ a, Amp *__restrict__ b,
                                                              uint64_t npairs, int q) {
    const uint64_t stride = (uint64_t)gridDim.x * kSwapThreads;
    const uint64_t low = (1ull << q) - 1ull, bit = 1ull << q;
    for (uint64_t g = blockIdx.x * (uint64_t)kSwapThreads + threadIdx.x; g < npairs; g += kSwapPer * stride) {
        Amp x[kSwapPer], y[kSwapPer];
        uint64_t idx[kSwapPer];
#pragma unroll
        for (int r = 0; r < kSwapPer; ++r) {
            const uint64_t gr = g + (uint64_t)r * stride;
            if (gr < npairs) {
                idx[r] = ((gr & ~low) << 1) | (gr & low);
                x[r] = a[idx[r] | bit];
                y[r] = b[idx[r]];
            }
        }
#pragma unroll
        for (int r = 0; r < kSwapPer; ++r) {
            const uint64_t gr = g + (uint64_t)r * stride;
            if (gr < npairs) {
                a[idx[r] | bit] = y[r];
                b[idx[r]] = x[r];
            }
        }
    }
}

}  // namespace

extern "C" {

int sim_swap_halves(qsim *a, qsim *b, int qubit) {
    if (!a || !b || a == b) return QSIM_EINVAL;
    if (a->n != b->n || a->prec != b->prec || a->device != b->device)
        return set_err(a, QSIM_EINVAL, "shards differ in size, precision or device");
    if (qubit < 0 || qubit >= a->n) return set_err(a, QSIM_ERANGE, "qubit index out of range");
    int rc = sim_flush(a);
    if (!rc) rc = sim_flush(b);
    if (rc) return rc;
    // b's queued work comes first, then the exchange on a's stream, then b
    // continues after it
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(a->stream, ev, 0);
    if (e != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        return cuda_err(a, e, "shard stream ordering");
    }
    const uint64_t npairs = 1ull << (a->n - 1);
    uint64_t grid = (npairs + (uint64_t)kSwapThreads * kSwapPer - 1) / ((uint64_t)kSwapThreads * kSwapPer);
    const uint64_t cap = (uint64_t)a->sms * 8;
    if (grid > cap) grid = cap;
    if (a->prec == QSIM_C128)
        k_swap_halves<double2><<<(unsigned)grid, kSwapThreads, 0, a->stream>>>((double2 *)a->state,
                                                                               (double2 *)b->state, npairs, qubit);
    else
        k_swap_halves<float2><<<(unsigned)grid, kSwapThreads, 0, a->stream>>>((float2 *)a->state,
                                                                              (float2 *)b->state, npairs, qubit);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev, a->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_err(a, e, "shard exchange launch");
    a->stats.launches++;
    a->stats.alg_bytes += 2.0 * (double)amp_bytes(a) * (double)npairs * 2.0;
    // both shards' norms changed: their block passes start new chains
    a->norm_chain = b->norm_chain = false;
    a->norm_target = b->norm_target = -1.0;
    return QSIM_OK;
}

int sim_project(qsim *s, const int *qubits, int m, const int *bits, double scale) {
    if (!s || m < 0 || (m > 0 && (!qubits || !bits))) return QSIM_EINVAL;
    if (!std::isfinite(scale)) return set_err(s, QSIM_ENONFINITE, "non-finite scale");
    uint64_t mask = 0, value = 0;
    for (int j = 0; j < m; ++j) {
        if (qubits[j] < 0 || qubits[j] >= s->n) return set_err(s, QSIM_ERANGE, "qubit index out of range");
        if ((mask >> qubits[j]) & 1ull) return set_err(s, QSIM_EDUP, "qubit named twice");
        if (bits[j] != 0 && bits[j] != 1) return set_err(s, QSIM_EINVAL, "bit values must be 0 or 1");
        mask |= 1ull << qubits[j];
        if (bits[j]) value |= 1ull << qubits[j];
    }
    int rc = sim_flush(s);
    if (rc) return rc;
    rc = run_collapse_mask(s, mask, value, scale);
    if (rc) return rc;
    s->norm_chain = false;
    s->norm_target = -1.0;
    return QSIM_OK;
}

}  // extern "C"

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
// moved[0] += sum |a[i | 2^q]|^2 (what leaves a), moved[1] += sum |b[i]|^2
// (what leaves b): FP32 within a round of kSwapPer pairs, FP64 beyond, one
// FP64 atomic per CTA.
template <typename Amp>
__global__ void __launch_bounds__(kSwapThreads) k_swap_halves(Amp *__restrict__ a, Amp *__restrict__ b,
                                                              uint64_t npairs, int q, double *moved) {
    typedef typename AmpTraits<Amp>::real R;
    const uint64_t stride = (uint64_t)gridDim.x * kSwapThreads;
    const uint64_t low = (1ull << q) - 1ull, bit = 1ull << q;
    double out_a = 0.0, out_b = 0.0;
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
        R sx = 0, sy = 0;
#pragma unroll
        for (int r = 0; r < kSwapPer; ++r) {
            const uint64_t gr = g + (uint64_t)r * stride;
            if (gr < npairs) {
                a[idx[r] | bit] = y[r];
                b[idx[r]] = x[r];
                sx += norm2(x[r]);
                sy += norm2(y[r]);
            }
        }
        out_a += (double)sx;
        out_b += (double)sy;
    }
    __shared__ double red[2][kSwapThreads / 32];
    out_a = warp_sum(out_a);
    out_b = warp_sum(out_b);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = out_a;
        red[1][threadIdx.x >> 5] = out_b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kSwapThreads / 32; ++w) {
            ta += red[0][w];
            tb += red[1][w];
        }
        atomicAdd(&moved[0], ta);
        atomicAdd(&moved[1], tb);
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
    double *moved = (double *)((char *)a->ws + kWsResult);
    e = cudaMemsetAsync(moved, 0, 2 * sizeof(double), a->stream);
    if (e == cudaSuccess) {
        if (a->prec == QSIM_C128)
            k_swap_halves<double2><<<(unsigned)grid, kSwapThreads, 0, a->stream>>>(
                (double2 *)a->state, (double2 *)b->state, npairs, qubit, moved);
        else
            k_swap_halves<float2><<<(unsigned)grid, kSwapThreads, 0, a->stream>>>(
                (float2 *)a->state, (float2 *)b->state, npairs, qubit, moved);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(a->pinned, moved, 2 * sizeof(double), cudaMemcpyDeviceToHost, a->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev, a->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_err(a, e, "shard exchange launch");
    a->stats.launches++;
    a->stats.alg_bytes += 2.0 * (double)amp_bytes(a) * (double)npairs * 2.0;
    // Both shards' norms changed by what moved.  Where both were known (the
    // targets of their norm control), the new ones are known too, so the
    // complex64 block passes keep steering to the exact norms and their
    // small per-chain errors cannot add up over many exchanges; otherwise
    // the next chains take their first pass's input norms.
    const double out_a = a->pinned[0], out_b = a->pinned[1];
    double ta = -1.0, tb = -1.0;
    if (a->norm_target >= 0.0 && b->norm_target >= 0.0) {
        ta = a->norm_target - out_a + out_b;
        tb = b->norm_target - out_b + out_a;
        if (ta < 0.0) ta = 0.0;
        if (tb < 0.0) tb = 0.0;
    }
    a->norm_chain = b->norm_chain = false;
    a->norm_target = ta;
    b->norm_target = tb;
    return QSIM_OK;
}

int sim_project(qsim *s, const int *qubits, int m, const int *bits, double scale, double kept_norm2) {
    if (!s || m < 0 || (m > 0 && (!qubits || !bits))) return QSIM_EINVAL;
    if (!std::isfinite(scale) || !std::isfinite(kept_norm2)) return set_err(s, QSIM_ENONFINITE, "non-finite scale");
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
    // the norm after the projection: scale^2 times what was kept, where
    // that is known (all of a known norm for m = 0, or the caller's figure)
    s->norm_chain = false;
    if (kept_norm2 >= 0.0)
        s->norm_target = scale * scale * kept_norm2;
    else if (m == 0 && s->norm_target >= 0.0)
        s->norm_target = scale * scale * s->norm_target;
    else
        s->norm_target = -1.0;
    return QSIM_OK;
}

}  // extern "C"

// noalloc.cu -- qsim_probs_all_noalloc: all single-qubit probabilities of a
// caller-owned state vector without any device allocation.
//
// Who needs this: callers that must not allocate GPU memory at the moment
// they ask for probabilities -- code that runs while another framework owns
// the whole device memory through its own pool (a cudaMalloc would fail or
// fragment that pool), real-time or embedded hosts with a fixed memory budget
// decided at start-up, and plugin hosts whose callbacks forbid allocation.
// The regular sim_probs_all path takes its scratch from the handle's
// workspace, which someone has to allocate; this entry point instead uses a
// fixed array compiled into the library.
//
// The scratch is a file-scope __device__ array of kScratchDoubles doubles
// (320 KiB: partial sums of up to 1024 CTAs for up to 36 qubits).  Every GPU
// that loads the library holds it until the process exits.  All calls share it: two calls whose kernels overlap on the GPU (for
// example on two streams) race on it and both results are undefined.  Each
// call overwrites every scratch entry it later reads, so nothing has to start
// at zero and the contents left by the previous call do not matter.
//
// In host code the symbol g_probs_scratch is only a host-side stand-in, not a
// device address; its device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, together with the
// device's SM count (the grid is four CTAs per SM, at most 1024).  The first
// call on a device does that set-up; make that first call before any stream
// capture.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1024;  // largest grid (four CTAs per SM)
constexpr int kNaMaxValues = 40;    // norm + up to 36 qubits, rounded up
constexpr int kScratchDoubles = kNaMaxBlocks * kNaMaxValues;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_probs_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
int g_grid_cap[kMaxDevices] = {0};

// Same tiling as the handle-based probabilities pass: a warp owns tiles of
// 1024 consecutive amplitudes, lane l reads index tile*1024 + 32*j + l.
template <typename Amp>
__global__ void __launch_bounds__(kNaThreads) k_na_probs_tiles(const Amp *__restrict__ psi, int n, uint64_t ntiles,
                                                               double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[kNaThreads / 32][2 * 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double accA = 0.0, accB = 0.0, accN = 0.0;
    for (uint64_t tile = (uint64_t)blockIdx.x * nw + warp; tile < ntiles; tile += (uint64_t)gridDim.x * nw) {
        const Amp *p = psi + (tile << 10) + lane;
        R S = 0, Sb[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const R w = norm2(p[j * 32]);
            S += w;
#pragma unroll
            for (int b = 0; b < 5; ++b)
                if ((j >> b) & 1) Sb[b] += w;
        }
        const double dS = (double)S;
        const double T = warp_sum(dS);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double a = warp_sum(((lane >> q) & 1) ? dS : 0.0);
            if (lane == q) accA += a;
        }
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const double a = warp_sum((double)Sb[b]);
            if (lane == 5 + b) accA += a;
        }
        const uint64_t base = tile << 10;
        if (lane >= 10 && lane < n && ((base >> lane) & 1ull)) accA += T;
        if (lane + 32 < n && ((base >> (lane + 32)) & 1ull)) accB += T;
        accN += T;
    }
    sh[warp][1 + lane] = accA;
    sh[warp][33 + lane] = accB;
    if (lane == 0) sh[warp][0] = accN;
    __syncthreads();
    const int V = n + 1;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sh[w][v];
        partials[(size_t)blockIdx.x * V + v] = t;
    }
}

// Registers below 10 qubits: one block, no scratch; writes the output.
template <typename Amp>
__global__ void k_na_probs_small(const Amp *__restrict__ psi, int n, double *__restrict__ out) {
    __shared__ double sh[32];
    const uint64_t N = 1ull << n;
    for (int v = 0; v <= n; ++v) {
        double acc = 0.0;
        for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) {
            const double w = (double)norm2(psi[i]);
            if (v == 0 || ((i >> (v - 1)) & 1ull)) acc += w;
        }
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
            out[v] = t;
        }
        __syncthreads();
    }
}

// Fixed-order second stage into the caller's output.
__global__ void k_na_finalize(const double *__restrict__ partials, int nblocks, int V, double *__restrict__ out) {
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partials[(size_t)b * V + v];
        out[v] = t;
    }
}

// Device address of the scratch array on the current device and the grid
// cap (looked up once per device).
int scratch_for_current_device(double **out, int *grid_cap) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QSIM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return QSIM_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        int sms = 0;
        cudaError_t e = cudaGetSymbolAddress(&p, g_probs_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || !p || sms < 1) {
            cudaGetLastError();
            return QSIM_ECUDA;
        }
        g_grid_cap[dev] = 4 * sms < kNaMaxBlocks ? 4 * sms : kNaMaxBlocks;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    *grid_cap = g_grid_cap[dev];
    return QSIM_OK;
}

template <typename Amp>
int probs_noalloc(const void *state, int n, double *out, cudaStream_t stream) {
    const Amp *psi = (const Amp *)state;
    if (n < 10) {
        k_na_probs_small<Amp><<<1, kNaThreads, 0, stream>>>(psi, n, out);
        return cudaGetLastError() == cudaSuccess ? QSIM_OK : QSIM_ECUDA;
    }
    double *scratch = nullptr;
    int cap = 0;
    int rc = scratch_for_current_device(&scratch, &cap);
    if (rc) return rc;
    const uint64_t ntiles = 1ull << (n - 10);
    const uint64_t want = (ntiles + (kNaThreads / 32) - 1) / (kNaThreads / 32);
    const int grid = (int)(want < (uint64_t)cap ? want : (uint64_t)cap);
    k_na_probs_tiles<Amp><<<grid, kNaThreads, 0, stream>>>(psi, n, ntiles, scratch);
    if (cudaGetLastError() != cudaSuccess) return QSIM_ECUDA;
    k_na_finalize<<<1, 64, 0, stream>>>(scratch, grid, n + 1, out);
    return cudaGetLastError() == cudaSuccess ? QSIM_OK : QSIM_ECUDA;
}

}  // namespace

extern "C" int qsim_probs_all_noalloc(const void *state, int n, int precision, double *out, void *stream) {
    if (!state || !out) return QSIM_EINVAL;
    if (precision != QSIM_C128 && precision != QSIM_C64) return QSIM_EINVAL;
    if (n < 1) return QSIM_EINVAL;
    if (n + 1 > kNaMaxValues || n > kMaxQubits) return QSIM_ENOTSUP;  // beyond the scratch array
    const uintptr_t align = precision == QSIM_C128 ? 16 : 8;
    if (((uintptr_t)state % align) || ((uintptr_t)out % 8)) return QSIM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    return precision == QSIM_C128 ? probs_noalloc<double2>(state, n, out, st)
                                  : probs_noalloc<float2>(state, n, out, st);
}

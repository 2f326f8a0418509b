// product_kernel.cu -- a layer of Hadamard-like one-qubit gates on many
// qubits, applied twelve qubits per pass over a complex64 state.
//
// The simulator executes buffered gates together (ProjectQ paper, Sec.
// 4.3.2).  Between gates too wide for any block (Grover's many-controlled Z,
// Appendix A) a layer of one-qubit gates on m qubits has nothing to fuse
// with; as dense 6-qubit blocks it costs ceil(m / 6) passes.  Grover's
// layers are products of H and X on each wire, c [[s00, s01], [s10, s11]]
// with c = 2^(-1/2), signs s = +-1 and orthogonal rows (s00 s11 = -s01
// s10), which the planner recognises ("butterfly" matrices).  For such a
// gate
//     x0' = c s00 (x0 + p x1),   x1' = c s10 (x0 - p x1),   p = s00 s01:
// two FMAs per amplitude, the factors c s00 / c s10 left for the end.  A
// pass takes tiles of 2^12 amplitudes whose bits V are the pass's qubits
// plus the lowest address bits (runs of at least 16 amplitudes, 128 bytes),
// applies the butterflies of all its qubits and multiplies each output once
// by C sigma (-1)^popc(e & F), C = prod c_j, sigma = prod s00_j, F = the
// tile bits whose s10 differs from s00: one read and one write of the
// state, about 40 instructions per amplitude.  (General complex 2x2 factors
// would cost 8 FMAs per amplitude and qubit, 96 for a 12-qubit pass, more
// than the issue rate allows at HBM speed; those layers stay with the
// tensor-core blocks.)
//
// A tile is 32 KB of shared memory, double-buffered: the next tile arrives
// by 16-byte cp.async copies (two amplitudes, bypassing L1) while this one
// is processed (64 KB per CTA, three CTAs per SM).  256 threads hold 16
// amplitudes each in three layouts (tile index e, bits 0..11):
//   A  e = i | tid << 4:                              registers = tile bits 0..3
//   B  e = (tid & 15) | i << 4 | (tid >> 4) << 8:     registers = tile bits 4..7
//   C  e = tid | i << 8:                              registers = tile bits 8..11
// The copies (e = 2 tid + i << 9, 16 bytes each) and the stores (layout C)
// put the lanes on the lowest tile bits (address bits 0..3 and more:
// 128-byte runs at least).  Element e sits at shared position
// e ^ ((e >> 4) & 7) << 1: bits 1..3 XOR bits 4..6, bit 0 kept, so an
// amplitude pair stays one aligned 16-byte slot; the 16-byte copies and
// layout-A accesses meet 8 different slots per quarter-warp and the 8-byte
// accesses of layouts B and C 16 different bank pairs per half-warp.  (A
// padded layout, rows of 16 with a pitch of 17, needs no address
// arithmetic per access but measured 5 % slower.)  The global addresses of
// a thread's copies and stores step through the register bits in Gray-code
// order, one 64-bit add each.
//
// Norm control.  A product pass is one step of the same norm chain as the
// tensor-core block passes (norm_chain.cuh): its inputs' and outputs' sums
// of |x|^2 per CTA in FP64 and the scale from the previous pass's record.
// C is rounded to FP32 (2^(-k/2) for k gates, exact only for even k) and the
// FP32 additions round; the control returns the norm to its target after
// every pass.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "norm_chain.cuh"

using namespace qsim_dev;

namespace {

constexpr int kPBits = 12;                           // tile bits
constexpr int kPThreads = 256;
constexpr int kPPer = (1 << kPBits) / kPThreads;     // amplitudes per thread: 16
constexpr int kPRegBits = 4;                         // log2(kPPer)
constexpr int kPCtasPerSm = 3;
constexpr int kPMinRun = 4;                          // runs of at least 2^4 amplitudes (128 B)
constexpr int kPTile = 1 << kPBits;                  // amplitudes per tile buffer
constexpr int kPSmem = 2 * kPTile * 8;               // two tile buffers (64 KB)

struct ProdArgs {
    float2 *psi;
    uint64_t ntiles;          // 2^(n - 12)
    InsertSpec vspec;         // the 12 tile bits V as address bits, ascending
    int nruns;                // V as runs of consecutive address bits: [run_pos, run_pos + run_len)
    int run_pos[kPBits];
    int run_len[kPBits];
    uint32_t gmask;           // tile bits that carry a gate
    uint32_t fmask;           // F: tile bits whose s10 differs from s00
    float p[kPBits];          // p = s00 s01 of tile bit j
    float cs;                 // C sigma
    qsim_chain::ChainArgs chain;  // norm control (norm_chain.cuh)
};

// shared-memory position of tile element e
__device__ __forceinline__ uint32_t swz(uint32_t e) { return e ^ (((e >> 4) & 7u) << 1); }

// Gray code of step k and the bit it changes from step k - 1
__host__ __device__ constexpr int gray(int k) { return k ^ (k >> 1); }
__host__ __device__ constexpr int gray_bit(int k) {
    if (k == 0) return -1;
    int b = 0;
    while (!((k >> b) & 1)) ++b;
    return b;
}

// First address of tile t: the bits of t spread around the runs of V
__device__ __forceinline__ uint64_t tile_base(uint64_t t, const ProdArgs &A) {
    for (int j = 0; j < A.nruns; ++j) {
        const int p = A.run_pos[j];
        t = ((t >> p) << (p + A.run_len[j])) | (t & ((1ull << p) - 1ull));
    }
    return t;
}

__device__ __forceinline__ void bfly(float2 &v0, float2 &v1, float p) {
    const float2 a = v0, b = v1;
    v0 = make_float2(fmaf(p, b.x, a.x), fmaf(p, b.y, a.y));
    v1 = make_float2(fmaf(-p, b.x, a.x), fmaf(-p, b.y, a.y));
}

// Butterflies of tile bits base + r (register bit r of the layout), for the
// r in `bits` (a 4-bit mask)
__device__ __forceinline__ void stage(float2 (&v)[kPPer], const ProdArgs &A, int base, uint32_t bits) {
#pragma unroll
    for (int r = 0; r < kPRegBits; ++r) {
        if (!((bits >> r) & 1u)) continue;
        const float p = A.p[base + r];
#pragma unroll
        for (int i = 0; i < kPPer; ++i)
            if (!((i >> r) & 1)) bfly(v[i], v[i | (1 << r)], p);
    }
}

// 16-byte asynchronous copy global -> shared (no register staging, not
// cached in L1)
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all of this thread's copies complete
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(kPThreads, kPCtasPerSm) k_product(const ProdArgs A) {
    extern __shared__ __align__(16) float2 smd[];  // two tiles of 2^12 amplitudes (positions swz(e))
    __shared__ float s_scale;
    __shared__ double s_red[kPThreads / 32][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // address bits of tile index e
    auto addr = [&](uint32_t e) {
        uint64_t a = 0;
#pragma unroll
        for (int j = 0; j < kPBits; ++j)
            if ((e >> j) & 1u) a |= 1ull << A.vspec.pos[j];
        return a;
    };
    if (tid == 0) s_scale = qsim_chain::chain_scale(A.chain);  // and the record
    __syncthreads();
    const float out_scale = s_scale * A.cs;  // every output, before its sign
    const uint64_t off_lo = addr((uint32_t)tid);          // tile bits 0..7 of this thread (stores)
    const uint64_t off_cp = addr((uint32_t)tid << 1);     // tile bits 1..8 of this thread's copies
    const uint32_t gA = A.gmask & 15u, gB = (A.gmask >> 4) & 15u, gC = (A.gmask >> 8) & 15u;
    // sign of output i (layout C, e = tid | i << 8) in bit i
    uint32_t sgn = 0;
    {
        const uint32_t f_tid = (uint32_t)__popc((uint32_t)tid & A.fmask) & 1u, f_hi = A.fmask >> 8;
#pragma unroll
        for (int i = 0; i < kPPer; ++i) sgn |= ((f_tid ^ (uint32_t)__popc((uint32_t)i & f_hi)) & 1u) << i;
    }
    // address bits of tile bits 8..11 (the register index of the copies and
    // of layout C)
    uint64_t hb[kPRegBits];
#pragma unroll
    for (int r = 0; r < kPRegBits; ++r) hb[r] = 1ull << A.vspec.pos[8 + r];
    // tile bits 9..11: the register index of the copies
    uint64_t cb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) cb[r] = 1ull << A.vspec.pos[9 + r];
    // layouts A (e = i | tid << 4) and B; C and the copies: e = tid | i << 8
    const uint32_t eA = (uint32_t)tid << 4, eB = ((uint32_t)tid & 15u) | (((uint32_t)tid >> 4) << 8);
    // copies of the tile at `base`: elements e, e + 1 with e = 2 tid + k << 9,
    // k in Gray order
    auto copy_in = [&](uint64_t base, int buf) {
        const float2 *p = A.psi + base + off_cp;
        float2 *d = smd + buf * kPTile;
#pragma unroll
        for (int k = 0; k < kPPer / 2; ++k) {
            const int g = gray(k), b = gray_bit(k);
            if (b >= 0) p = (gray(k - 1) >> b) & 1 ? p - cb[b] : p + cb[b];
            cp_async16(d + swz(((uint32_t)tid << 1) | ((uint32_t)g << 9)), p);
        }
    };
    double nin = 0.0, nout = 0.0;
    uint64_t t = blockIdx.x;
    uint64_t base = t < A.ntiles ? tile_base(t, A) : 0;
    if (t < A.ntiles) copy_in(base, 0);
    cp_async_commit();
    for (int it = 0; t < A.ntiles; t += gridDim.x, ++it) {
        cp_async_wait_all();
        // every thread's copies of tile t have landed, and every thread is
        // done with iteration it - 1, whose buffer the next copies refill
        __syncthreads();
        const uint64_t tn = t + gridDim.x;
        const uint64_t base_n = tn < A.ntiles ? tile_base(tn, A) : 0;
        if (tn < A.ntiles) copy_in(base_n, (it + 1) & 1);  // in flight during this tile's stages
        cp_async_commit();
        float2 *x = smd + (it & 1) * kPTile;
        float2 v[kPPer];
        // layout A: input sums, butterflies of tile bits 0..3
        {
#pragma unroll
            for (int j = 0; j < kPPer / 2; ++j) {
                const float4 w = *(const float4 *)(x + swz(eA | 2u * (uint32_t)j));
                v[2 * j] = make_float2(w.x, w.y);
                v[2 * j + 1] = make_float2(w.z, w.w);
            }
            float q[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < kPPer; ++i) q[i & 3] = fmaf(v[i].x, v[i].x, fmaf(v[i].y, v[i].y, q[i & 3]));
            nin += (double)((q[0] + q[1]) + (q[2] + q[3]));
            if (gA) {
                stage(v, A, 0, gA);
#pragma unroll
                for (int j = 0; j < kPPer / 2; ++j)
                    *(float4 *)(x + swz(eA | 2u * (uint32_t)j)) =
                        make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
            }
            __syncthreads();
        }
        if (gB) {
            // layout B: butterflies of tile bits 4..7
#pragma unroll
            for (int i = 0; i < kPPer; ++i) v[i] = x[swz(eB | ((uint32_t)i << 4))];
            stage(v, A, 4, gB);
#pragma unroll
            for (int i = 0; i < kPPer; ++i) x[swz(eB | ((uint32_t)i << 4))] = v[i];
            __syncthreads();
        }
        // layout C: butterflies of tile bits 8..11, the output factors,
        // output sums, stores
#pragma unroll
        for (int i = 0; i < kPPer; ++i) v[i] = x[swz((uint32_t)tid | ((uint32_t)i << 8))];
        stage(v, A, 8, gC);
        {
            float q[4] = {0.f, 0.f, 0.f, 0.f};
            float2 *p = A.psi + base + off_lo;
#pragma unroll
            for (int k = 0; k < kPPer; ++k) {
                const int i = gray(k), b = gray_bit(k);
                if (b >= 0) p = (gray(k - 1) >> b) & 1 ? p - hb[b] : p + hb[b];
                q[k & 3] = fmaf(v[i].x, v[i].x, fmaf(v[i].y, v[i].y, q[k & 3]));
                const float f = ((sgn >> i) & 1u) ? -out_scale : out_scale;
                *p = make_float2(v[i].x * f, v[i].y * f);
            }
            nout += (double)((q[0] + q[1]) + (q[2] + q[3]));
        }
        base = base_n;
    }
    // per-CTA sums, fixed order; the outputs' sum before the chain's scale
    nin = warp_sum(nin);
    nout = warp_sum(nout);
    if (lane == 0) {
        s_red[warp][0] = nin;
        s_red[warp][1] = nout;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kPThreads / 32; ++w) {
            a += s_red[w][0];
            b += s_red[w][1];
        }
        qsim_chain::chain_sums(A.chain, a, b * (double)A.cs * (double)A.cs);
    }
}

// One pass: the butterfly gates of `qubits` (m of them, ascending, at most
// 12) with tile bits V = qubits plus the lowest address bits outside them.
int launch_pass(qsim *s, const int *qubits, const cd *const *mats, int m) {
    const int n = s->n;
    ProdArgs a{};
    uint64_t V = 0;
    for (int j = 0; j < m; ++j) V |= 1ull << qubits[j];
    for (int b = 0; b < n && __builtin_popcountll(V) < kPBits; ++b) V |= 1ull << b;
    a.vspec.m = kPBits;
    double C = 1.0, sigma = 1.0;
    for (int b = 0, k = 0; b < n; ++b)
        if ((V >> b) & 1ull) {
            for (int j = 0; j < m; ++j)
                if (qubits[j] == b) {
                    const cd *u = mats[j];
                    if (!butterfly2(u)) return set_err(s, QSIM_EINVAL, "product pass: not a butterfly matrix");
                    const double s00 = u[0].real() > 0 ? 1.0 : -1.0, s01 = u[1].real() > 0 ? 1.0 : -1.0,
                                 s10 = u[2].real() > 0 ? 1.0 : -1.0;
                    a.p[k] = (float)(s00 * s01);
                    if (s10 != s00) a.fmask |= 1u << k;
                    a.gmask |= 1u << k;
                    C *= std::abs(u[0]);
                    sigma *= s00;
                }
            a.vspec.pos[k++] = b;
        }
    a.cs = (float)(C * sigma);
    for (int k = 0; k < kPBits;) {
        int l = 1;
        while (k + l < kPBits && a.vspec.pos[k + l] == a.vspec.pos[k] + l) ++l;
        a.run_pos[a.nruns] = a.vspec.pos[k];
        a.run_len[a.nruns++] = l;
        k += l;
    }
    a.psi = (float2 *)s->state;
    a.ntiles = 1ull << (n - kPBits);
    uint64_t cap = (uint64_t)s->sms * kPCtasPerSm;
    if (cap > (uint64_t)kMaxTcGrid) cap = kMaxTcGrid;
    const uint64_t grid = a.ntiles < cap ? a.ntiles : cap;
    a.chain = qsim_chain::chain_next(s);  // the norm chain of the block passes
    static bool attr_set[64] = {false};
    if (s->device < 0 || s->device >= 64) return QSIM_ENOTSUP;
    if (!attr_set[s->device]) {
        const cudaError_t e = cudaFuncSetAttribute(k_product, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
        if (e != cudaSuccess) return cuda_err(s, e, "product pass attribute");
        attr_set[s->device] = true;
    }
    k_product<<<(unsigned)grid, kPThreads, kPSmem, s->stream>>>(a);
    s->stats.launches++;
    qsim_chain::chain_advance(s, (int)grid);
    return cuda_err(s, cudaGetLastError(), "product pass launch");
}

}  // namespace

int product_pass_count(uint64_t qmask) {
    const uint64_t low = qmask & ((1ull << kPBits) - 1ull);
    const int nlo = __builtin_popcountll(low), nhi = __builtin_popcountll(qmask >> kPBits);
    const int per = kPBits - kPMinRun;
    const int npass_hi = (nhi + per - 1) / per;
    const int last = nhi - (npass_hi - 1) * per;
    const int top_lo = low ? 63 - __builtin_clzll(low) : -1;
    const bool fold = npass_hi > 0 && (nlo == 0 || top_lo < kPBits - last);
    return npass_hi + ((nlo > 0 && !fold) ? 1 : 0);
}

int launch_product(qsim *s, uint64_t qmask, const cd *mats, int *npasses) {
    *npasses = 0;
    if (s->prec != QSIM_C64 || s->n < kPBits) return QSIM_ENOTSUP;
    int lo[64], hi[64], nlo = 0, nhi = 0;
    const cd *mlo[64], *mhi[64];
    for (int b = 0, k = 0; b < s->n; ++b)
        if ((qmask >> b) & 1ull) {
            if (b < kPBits) {
                mlo[nlo] = mats + 4 * k;
                lo[nlo++] = b;
            } else {
                mhi[nhi] = mats + 4 * k;
                hi[nhi++] = b;
            }
            ++k;
        }
    // the qubits above the tile, kPBits - kPMinRun per pass; the last (the
    // smallest) pass also takes the low qubits if they lie in its runs
    const int per = kPBits - kPMinRun;
    const int npass_hi = (nhi + per - 1) / per;
    const int last = nhi - (npass_hi - 1) * per;  // qubits of the last high pass
    const bool fold = npass_hi > 0 && (nlo == 0 || lo[nlo - 1] < kPBits - last);
    int rc = QSIM_OK;
    if (nlo > 0 && !fold) {
        rc = launch_pass(s, lo, mlo, nlo);
        ++*npasses;
    }
    for (int p = 0; p < npass_hi && !rc; ++p) {
        int q[kPBits];
        const cd *m[kPBits];
        int k = 0;
        if (p == npass_hi - 1 && fold)
            for (int j = 0; j < nlo; ++j) {
                q[k] = lo[j];
                m[k++] = mlo[j];
            }
        for (int j = p * per; j < nhi && j < (p + 1) * per; ++j) {
            q[k] = hi[j];
            m[k++] = mhi[j];
        }
        rc = launch_pass(s, q, m, k);
        ++*npasses;
    }
    return rc;
}

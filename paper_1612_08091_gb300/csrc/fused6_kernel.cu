// fused6_kernel.cu -- a fused 6-qubit block applied on the tensor cores
// (tcgen05 / TMEM), complex64 amplitudes, BF16x3 split products.
//
// The same method as the 5-qubit kernel (fused_kernel.cu: lazily buffered
// gates executed together, ProjectQ paper Sec. 4.3.2, Fig. 7 caption), one
// qubit wider.  A run of gates on the 6 qubits S = {s0 < ... < s5} has been
// multiplied into one 64 x 64 complex matrix U, and the pass computes
// Psi' = U Psi with Psi viewed as a 64 x 2^(n-6) matrix.  A wider block takes
// more gates per pass over the state (a depth-40 brickwork on 32 qubits needs
// 69 passes with 6-qubit blocks against 106 with 5-qubit ones) for twice the
// tensor work per amplitude: 1536 flop per 16 bytes moved, still well below
// the bf16 ridge of this part (about 286 flop per byte).
//
// GEMM per tile of 128 columns: D(128 x 128) = X(128 x 128) R^T(128 x 128),
// M = 128 tile columns (the 7 lowest qubits F outside S), N = K = 128 (the
// real form of 64 complex rows, R[2r+a][2r'+b] the 2x2 real block of
// U[r][r']).  A tile is the 2^13 amplitudes whose bits outside V = S u F are
// fixed.
//
// Where the operands live.  R, split into two (or three) bf16 parts, is
// operand B in shared memory: K-major, 128-byte swizzle, as two 64-element K
// halves of 16 KB per part.  The state tile X is operand A and lives in
// tensor memory: thread t owns tile column t, which is TMEM lane t; it loads
// that column's 64 amplitudes, splits each into bf16 hi and lo words (re in
// the low half: K elements 2r, 2r+1) and writes them with tcgen05.st to TMEM
// columns [0, 64) (hi) and [64, 128) (lo).  The accumulator takes columns
// [128, 256).  So the state is never staged in shared memory and needs no
// swizzle arithmetic, and a CTA holds 256 TMEM columns and ~66 KB of shared
// memory: two CTAs per SM.
//
// Per CTA, over its tiles t of a persistent grid:
//   wait for MMA(t-1) -> read D(t-1) from TMEM, scale, store it -> split tile
//   t into TMEM -> thread 0 issues 24 (or 40) tcgen05.mma M128 N128 K16 and
//   commits them to an mbarrier -> issue the loads of tile t+1 (64
//   amplitudes per thread held in registers: 128 KB in flight per SM).
// The other CTA on the SM fills this CTA's waits.  Norm tracking is the
// 5-qubit kernel's: per-CTA FP64 sums of |x|^2 and |y|^2, and the outputs
// scaled by sqrt(in/out) of the previous block pass (of either kernel).
// Every wait is bounded; on time-out the kernel raises an error flag in the
// workspace, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

using namespace qsim_dev;
using namespace qsim_tc;

namespace {

constexpr int kT6Threads = 128;
constexpr int kT6TileBits = 13;           // 6 row bits + 7 column bits
constexpr int kB6Half = 128 * 128;        // one K half of one bf16 part of R: 128 rows x 128 B
constexpr int kB6Bytes = 2 * kB6Half;     // one bf16 part of R (128 x 128)
constexpr uint32_t kT6Cols = 256;         // TMEM columns per CTA
constexpr uint32_t kColAHi = 0, kColALo = 64, kColD = 128;
constexpr uint32_t kIdesc6 = idesc_bf16(128, 128);
constexpr int kT6Extra = 128;             // barriers, TMEM slot, flags, reduction

struct Tc6Args {
    float2 *psi;
    const unsigned char *rec;  // nsplit x kB6Bytes: pre-split, pre-swizzled R (16-B aligned)
    uint32_t rec_bytes;
    int nsplit;                // bf16 parts of R: 2 (BF16x3) or 3 (five products)
    uint64_t ntiles;           // 2^(n-13)
    InsertSpec vspec;          // the 13 positions of V = S u F, ascending
    unsigned int *err;         // error flag
    double *norm_out;          // this pass's per-CTA sums (see the 5-qubit kernel)
    const double *norm_prev;   // the previous block pass's sums, or null
    int prev_grid;
    int fpos[7];               // tile column bit j <-> qubit fpos[j]
    uint64_t rdep[64];         // address bits of block row r
};

// D(tmem) (+)= A(tmem) * B(smem)^T, M = N = 128, K = 16
__device__ __forceinline__ void mma6(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(kIdesc6), "r"(accumulate)
        : "memory");
}

// PAIR: qubit 0 is in S, so rows r and r+1 (r even) are adjacent amplitudes
// and move as one 16-byte access.
template <bool PAIR>
__global__ void __launch_bounds__(kT6Threads, 2) k_block_tc6(const Tc6Args args) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *B = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(B + args.nsplit * kB6Bytes);  // [0] operand copy, [1] MMA done
    uint32_t *tmem_slot = (uint32_t *)(bars + 2);
    float *s_scale = (float *)(tmem_slot + 1);
    double *s_red = (double *)(bars + 4);  // [4 warps][2]

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // output scale from the previous pass's input/output norms, summed
        // in a fixed order
        float sc = 1.0f;
        if (args.norm_prev) {
            double a = 0.0, b = 0.0;
            for (int i = 0; i < args.prev_grid; ++i) {
                a += args.norm_prev[i];
                b += args.norm_prev[kMaxTcGrid + i];
            }
            if (a > 0.0 && b > 0.0 && a < 1e300 && b < 1e300) sc = (float)sqrt(a / b);
        }
        *s_scale = sc;
    }
    __syncthreads();
    if (tid == 0) bulk_load(B, args.rec, args.rec_bytes, &bars[0]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kT6Cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 TMEM lanes

    bool failed = !mbar_wait(&bars[0], 0);
    if (failed) atomicOr(args.err, 1u);
    const bool abort0 = __syncthreads_or(failed) != 0;

    double nrm_in = 0.0, nrm_out = 0.0;
    const float scale = *s_scale;
    if (!abort0) {
        uint64_t coff = 0;  // address bits of this thread's tile column
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if ((tid >> j) & 1) coff |= 1ull << args.fpos[j];
        const int nterms = args.nsplit == 3 ? 5 : 3;

        float4 v[32];  // rows 2j, 2j+1 of this column: (re, im, re, im)
        auto load_tile = [&](uint64_t tt) {
            const float2 *p = args.psi + insert_zeros(tt, args.vspec) + coff;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (PAIR) {
                    v[j] = *(const float4 *)(p + args.rdep[2 * j]);
                } else {
                    const float2 a = p[args.rdep[2 * j]], b = p[args.rdep[2 * j + 1]];
                    v[j] = make_float4(a.x, a.y, b.x, b.y);
                }
            }
        };
        auto epilogue = [&](uint64_t tt) {
            float2 *p = args.psi + insert_zeros(tt, args.vspec) + coff;
            float ssq = 0.f;
#pragma unroll
            for (int chunk = 0; chunk < 4; ++chunk) {
                float d[32];  // rows 16 chunk .. 16 chunk + 15, (re, im) interleaved
                tmem_ld32(lanes + kColD + chunk * 32, d);
#pragma unroll
                for (int q = 0; q < 32; ++q) ssq = fmaf(d[q], d[q], ssq);
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const int r = chunk * 16 + q;
                    if (PAIR) {
                        *(float4 *)(p + args.rdep[r]) = make_float4(d[2 * q] * scale, d[2 * q + 1] * scale,
                                                                     d[2 * q + 2] * scale, d[2 * q + 3] * scale);
                    } else {
                        p[args.rdep[r]] = make_float2(d[2 * q] * scale, d[2 * q + 1] * scale);
                        p[args.rdep[r + 1]] = make_float2(d[2 * q + 2] * scale, d[2 * q + 3] * scale);
                    }
                }
            }
            nrm_out += (double)ssq;
        };

        uint64_t t = blockIdx.x;
        int it = 0;
        bool stop = false;
        if (t < args.ntiles) load_tile(t);
        for (; t < args.ntiles; t += gridDim.x, ++it) {
            if (it >= 1) {
                // MMA(it-1) done: the A columns are free and D holds the
                // previous tile
                if (mbar_wait(&bars[1], (uint32_t)((it - 1) & 1))) {
                    tc_fence_after();
                    epilogue(t - gridDim.x);
                } else {
                    failed = true;
                    atomicOr(args.err, 2u);
                }
            }
            float xsq = 0.f;
#pragma unroll
            for (int chunk = 0; chunk < 4; ++chunk) {
                uint32_t hw[16], lw[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 x = v[chunk * 8 + j];
                    xsq = fmaf(x.x, x.x, fmaf(x.y, x.y, xsq));
                    xsq = fmaf(x.z, x.z, fmaf(x.w, x.w, xsq));
                    split_pair(x.x, x.y, hw[2 * j], lw[2 * j]);
                    split_pair(x.z, x.w, hw[2 * j + 1], lw[2 * j + 1]);
                }
                tmem_st16(lanes + kColAHi + chunk * 16, hw);
                tmem_st16(lanes + kColALo + chunk * 16, lw);
            }
            nrm_in += (double)xsq;
            tcgen05_wait_st();
            tc_fence_before();
            if (__syncthreads_or(failed)) {
                stop = true;
                break;
            }
            if (tid == 0) {
                tc_fence_after();
                const uint32_t b0 = smem_u32(B);
                uint32_t acc = 0;
                for (int term = 0; term < nterms; ++term) {
                    // (A part, B part): X1R1, X2R1, X1R2, X2R2, X1R3
                    const uint32_t a = tmem + ((term == 1 || term == 3) ? kColALo : kColAHi);
                    const uint32_t b = b0 + (uint32_t)(term < 2 ? 0 : (term < 4 ? 1 : 2)) * kB6Bytes;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        mma6(tmem + kColD, a + kk * 8, sw128_desc(b + (kk >> 2) * kB6Half + (kk & 3) * 32), acc);
                        acc = 1;
                    }
                }
                mma_commit(&bars[1]);
            }
            const uint64_t tn = t + gridDim.x;
            if (tn < args.ntiles) load_tile(tn);
        }
        if (it >= 1 && !stop) {
            if (mbar_wait(&bars[1], (uint32_t)((it - 1) & 1))) {
                tc_fence_after();
                epilogue(t - gridDim.x);
            } else {
                atomicOr(args.err, 2u);
            }
        }
    }
    // per-CTA norm sums, fixed reduction order
    nrm_in = warp_sum(nrm_in);
    nrm_out = warp_sum(nrm_out);
    if ((tid & 31) == 0) {
        s_red[2 * warp] = nrm_in;
        s_red[2 * warp + 1] = nrm_out;
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && args.norm_out) {
        args.norm_out[blockIdx.x] = s_red[0] + s_red[2] + s_red[4] + s_red[6];
        args.norm_out[kMaxTcGrid + blockIdx.x] = s_red[1] + s_red[3] + s_red[5] + s_red[7];
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kT6Cols) : "memory");
    }
}

// The B operand image: the nsplit bf16 parts of R = real form of U, each
// 128 rows (output index 2r+a) x 128 K elements (input index 2r'+b) in two K
// halves of 64 elements; within a half, row `row` is 128 bytes at row * 128
// with its 16-byte chunks XOR-swizzled by row & 7.
void build_operand6(const cd *U, int nsplit, std::vector<unsigned char> &rec) {
    rec.assign((size_t)nsplit * kB6Bytes, 0);
    for (int row = 0; row < 128; ++row)
        for (int k = 0; k < 128; ++k) {
            const cd u = U[(row >> 1) * 64 + (k >> 1)];
            const int a = row & 1, b = k & 1;
            double rem = a == 0 ? (b == 0 ? u.real() : -u.imag()) : (b == 0 ? u.imag() : u.real());
            const int kb = (k & 63) * 2;
            const size_t off =
                (size_t)(k >> 6) * kB6Half + (size_t)row * 128 + ((((kb >> 4) ^ (row & 7)) << 4)) + (kb & 15);
            for (int sp = 0; sp < nsplit; ++sp) {
                const uint16_t h = f32_to_bf16_bits((float)rem);
                rem -= bf16_bits_to_double(h);
                std::memcpy(&rec[(size_t)sp * kB6Bytes + off], &h, 2);
            }
        }
}

}  // namespace

int launch_block_tc6(qsim *s, const int *qubits, const cd *m) {
    if (s->prec != QSIM_C64 || s->n < kT6TileBits || !s->tc_enabled) return QSIM_ENOTSUP;
    const int n = s->n;
    const int nsplit = s->tc_terms == 5 ? 3 : 2;
    Tc6Args a{};
    uint64_t Smask = 0;
    for (int j = 0; j < 6; ++j) Smask |= 1ull << qubits[j];
    uint64_t Vmask = Smask;
    for (int b = 0, nf = 0; b < n && nf < 7; ++b)
        if (!((Smask >> b) & 1ull)) {
            a.fpos[nf++] = b;
            Vmask |= 1ull << b;
        }
    a.vspec.m = kT6TileBits;
    for (int b = 0, k = 0; b < n; ++b)
        if ((Vmask >> b) & 1ull) a.vspec.pos[k++] = b;
    for (int r = 0; r < 64; ++r) {
        uint64_t d = 0;
        for (int j = 0; j < 6; ++j)
            if ((r >> j) & 1) d |= 1ull << qubits[j];
        a.rdep[r] = d;
    }
    const bool pair = qubits[0] == 0;

    std::vector<unsigned char> rec;
    build_operand6(m, nsplit, rec);
    unsigned char *dev_rec = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev_rec);
    if (rc) return rc;

    auto kernel = pair ? k_block_tc6<true> : k_block_tc6<false>;
    const int dev = s->device;
    if (dev < 0 || dev >= 64) return QSIM_ENOTSUP;
    static int smem_for[2][64][4] = {{{0}}};  // [pair][device][nsplit]: dynamic shared memory to request
    int &smem = smem_for[pair ? 1 : 0][dev][nsplit];
    if (!smem) {
        // Two CTAs per SM: the tensor memory holds two 256-column CTAs.  If
        // registers and shared memory would let a third CTA in, request more
        // shared memory so that it stays out (its allocation would wait for
        // one of the others to finish and unbalance the persistent grid).
        cudaFuncAttributes fa;
        int regs_sm = 65536, smem_sm = 233472;
        cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return cuda_err(s, e, "tc6 kernel attributes");
        int bytes = 1024 + nsplit * kB6Bytes + kT6Extra;
        const int by_regs = regs_sm / (fa.numRegs * kT6Threads);
        if (by_regs >= 3 && smem_sm / (bytes + 1024) >= 3) bytes = smem_sm / 3 - 1024 + 64;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return cuda_err(s, e, "tc6 kernel attribute");
        if (getenv("QSIM_DEBUG"))
            fprintf(stderr, "qsim: k_block_tc6<%d> regs %d smem %d (registers allow %d CTAs/SM)\n", pair ? 1 : 0,
                    fa.numRegs, bytes, by_regs);
        smem = bytes;
    }
    a.psi = (float2 *)s->state;
    a.rec = dev_rec;
    a.rec_bytes = (uint32_t)rec.size();
    a.nsplit = nsplit;
    a.ntiles = 1ull << (n - kT6TileBits);
    a.err = (unsigned int *)((char *)s->ws + kWsErr);
    const uint64_t cap = (uint64_t)kSMs * 2;
    const uint64_t grid = a.ntiles < cap ? a.ntiles : cap;
    double *slots = (double *)((char *)s->ws + kWsNorm);
    const int slot = (int)(s->tc_passes & 1);
    a.norm_out = slots + slot * 2 * kMaxTcGrid;
    a.norm_prev = (s->norm_tracking && s->tc_passes > 0) ? slots + (slot ^ 1) * 2 * kMaxTcGrid : nullptr;
    a.prev_grid = s->tc_prev_grid;
    kernel<<<(unsigned)grid, kT6Threads, smem, s->stream>>>(a);
    s->stats.launches++;
    s->tc_passes++;
    s->tc_prev_grid = (int)grid;
    return cuda_err(s, cudaGetLastError(), "tc6 block launch");
}

// tmem_block_kernel.cu -- a fused 5- or 6-qubit block applied on the tensor
// cores (tcgen05) with the state operand in tensor memory; complex64
// amplitudes, BF16x3 split products.
//
// The paper's simulator gains its speed from lazily buffering gates and
// executing them together (ProjectQ paper, Sec. 4.3.2, Fig. 7 caption).
// Here a run of gates on the K qubits S = {s0 < ... < s(K-1)} (K = 5 or 6)
// has been multiplied into one 2^K x 2^K complex matrix U, and the pass
// computes Psi' = U Psi with Psi viewed as a 2^K x 2^(n-K) matrix (row = the
// bits of S).  A 6-qubit block takes more gates per pass over the state (a
// depth-40 brickwork on 32 qubits needs 69 passes with 6-qubit blocks
// against 106 with 5-qubit ones) for twice the tensor work per amplitude:
// 1536 flop per 16 bytes moved, still well below the bf16 ridge of this part
// (about 286 flop per byte).
//
// Real form.  With interleaved (re, im) amplitudes, the real vector x of a
// column (x[2r] = Re psi_r, x[2r+1] = Im psi_r) maps to y = R x with
// R[2r+a][2r'+b] the 2x2 real block of U[r][r'].  A tile of 128 columns is
// the GEMM D(128 x N) = X(128 x N) R^T(N x N), N = 2^(K+1): M = 128 tile
// columns (the 7 lowest qubits F outside S), N = K_mma = the real form of
// the 2^K rows.  A tile is the 2^(K+7) amplitudes whose bits outside
// V = S u F are fixed.
//
// BF16x3.  X = X1 + X2 and R = R1 + R2 (+ R3) are split into bfloat16 parts;
// the products X1 R1 + X2 R1 + X1 R2 (or five with X2 R2 + X1 R3) accumulate
// in FP32 in tensor memory.  The state split loses about 2^-17 relatively
// per element and pass; the gate split is computed on the host in FP64.
//
// Where the operands live.  R's bf16 parts are operand B in shared memory:
// K-major, 128-byte swizzle, in 64-element K halves of N x 128 bytes.  The
// state tile X is operand A and lives in tensor memory: thread t owns tile
// column t, which is TMEM lane t; it loads that column's 2^K amplitudes,
// splits each into bf16 hi and lo words (re in the low half: K elements 2r,
// 2r+1) and writes them with tcgen05.st to TMEM columns [0, 2^K) (hi) and
// [2^K, 2^(K+1)) (lo); the accumulator takes the next N columns.  So the
// state is never staged in shared memory and needs no swizzle arithmetic.
// Per CTA: 2^(K+2) TMEM columns (128 or 256) and 17 or 66 KB of shared
// memory; three (K = 5) or two (K = 6) CTAs per SM.
//
// Per CTA, over its tiles t of a persistent grid:
//   wait for MMA(t-1) -> read D(t-1) from TMEM, scale, store it -> split tile
//   t into TMEM -> thread 0 issues N/16 tcgen05.mma M128 N K16 per product
//   and commits them to an mbarrier -> issue the loads of tile t+1 (2^K
//   amplitudes per thread held in registers: 96 or 128 KB in flight per SM).
// The other CTAs on the SM fill this CTA's waits.  Every wait is bounded; on
// time-out the kernel raises an error flag in the workspace, frees its
// tensor memory and returns.
//
// Norm control.  The bf16 split and the FP32 accumulation shrink the norm by
// a few 1e-7 per pass, and the shrink is systematic on structured states
// (Grover's search repeats the same blocks on a state whose amplitudes are
// mostly equal), so uncorrected it adds up over 1e5 passes.  Each pass is a
// step of the norm chain of norm_chain.cuh: from the previous pass's input
// and output sums it scales its outputs so that the norm returns to the
// chain's target.  Errors therefore do not accumulate: what remains is one
// pass's change of shrink ratio and the drift of the passes outside the
// chain since the previous one, both corrected by the pass after.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "norm_chain.cuh"
#include "tc_common.cuh"

using namespace qsim_dev;
using namespace qsim_tc;

namespace {

constexpr int kTmThreads = 128;
constexpr int kTmExtra = 128;  // barriers, TMEM slot, scale, reduction

template <int K>
struct TmShape {
    static constexpr int kRows = 1 << K;          // block rows
    static constexpr int kTileBits = K + 7;       // + 7 column bits
    static constexpr int kN = 2 * kRows;          // real outputs = real inputs
    static constexpr int kBHalf = kN * 128;       // one 64-element K half of one part: N rows x 128 B
    static constexpr int kBPart = (kN / 64) * kBHalf;
    static constexpr uint32_t kColAHi = 0, kColALo = kRows, kColD = 2 * kRows;
    static constexpr uint32_t kCols = 4 * kRows;  // tensor-memory columns per CTA
    static constexpr uint32_t kIdesc = idesc_bf16(128, kN);
    static constexpr int kCtasPerSm = 512 / kCols < 3 ? 512 / kCols : 3;
};

struct TmArgs {
    float2 *psi;
    const unsigned char *rec;  // nsplit x kBPart: pre-split, pre-swizzled R (16-B aligned)
    uint32_t rec_bytes;
    int nsplit;                // bf16 parts of R: 2 (BF16x3) or 3 (five products)
    uint64_t ntiles;           // 2^(n - K - 7)
    InsertSpec vspec;          // the K + 7 positions of V = S u F, ascending
    unsigned int *err;         // error flag
    qsim_chain::ChainArgs chain;  // norm control (norm_chain.cuh)
    int fpos[7];               // tile column bit j <-> qubit fpos[j]
    uint64_t rdep[64];         // address bits of block row r
    uint64_t qoff[4];          // W = 16: address bits of column 4q + i relative to column 4q
};

// 32-byte global accesses (one whole sector per thread): four adjacent
// amplitudes as two float4 (the address is 32-byte aligned)
__device__ __forceinline__ void ld_v8(const float2 *p, float4 &a, float4 &b) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}
__device__ __forceinline__ void st_v8(float2 *p, const float4 &a, const float4 &b) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// D(tmem) (+)= A(tmem) * B(smem)^T, M = 128, K = 16
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// W: amplitudes per global access.  W = 2: qubit 0 is in S, so rows r and
// r+1 (r even) are adjacent amplitudes and move as one 16-byte access.  W = 4:
// qubits 0 and 1 are in S, rows 4j..4j+3 are adjacent and move as one
// 32-byte access; the tile columns are then at least 4 amplitudes apart, and
// narrower accesses would use half a sector per instruction.  W = 1: 8-byte
// accesses, the columns being adjacent amplitudes.  W = 16: qubits 0..3 are
// in S, so each 16-row line of a column is 128 contiguous bytes, but the
// lanes' columns lie 512 (K = 6) or 256 (K = 5) bytes apart and a warp
// access with one column per lane touches 32 lines.  Instead the four lanes
// of a quad read one column's line together (32 bytes each: 8 lines per
// warp access) and move it to and from tensor memory with the 16x256b
// shape, in which a quad shares a TMEM lane and each of its threads holds
// two adjacent 32-bit columns per 8.  Thread k of a quad holds rows 4k..4k+3
// of each 16-row line; the host orders the gate operand's K (input rows)
// and N (output rows) to match: A column 16G + 8h + 2k + e holds row
// 16G + 4k + 2h + e, and D columns 2j, 2j + 1 with j = 16G + 4h + k hold
// output row 16G + 4k + h.  Tile column 32w + q + 8i (warp w, quad q) is
// TMEM lane 32w + q + 8i as in the other widths.
template <int K, int W>
__global__ void __launch_bounds__(kTmThreads, TmShape<K>::kCtasPerSm) k_block_tmem(const TmArgs args) {
    using Sh = TmShape<K>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *B = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(B + args.nsplit * Sh::kBPart);  // [0] operand copy, [1] MMA done
    uint32_t *tmem_slot = (uint32_t *)(bars + 2);
    float *s_scale = (float *)(tmem_slot + 1);
    double *s_red = (double *)(bars + 4);  // [4 warps][2]

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // output scale from the previous pass's sums, and record
        *s_scale = qsim_chain::chain_scale(args.chain);
    }
    __syncthreads();
    if (tid == 0) bulk_load(B, args.rec, args.rec_bytes, &bars[0]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(Sh::kCols)
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
        // W = 16: this lane's place k4 in its quad q4; the address bits of
        // the quad's first column 32 warp + q4 (the others: + qoff[i])
        const unsigned lane = (unsigned)tid & 31u, k4 = lane & 3u, q4 = lane >> 2;
        uint64_t coffq = 0;
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if ((((tid & ~31) | (int)q4) >> j) & 1) coffq |= 1ull << args.fpos[j];
        const int nterms = args.nsplit == 3 ? 5 : 3;

        float4 v[Sh::kRows / 2];  // rows 2j, 2j+1 of this column: (re, im, re, im)
        auto load_tile = [&](uint64_t tt) {
            const float2 *p = args.psi + insert_zeros(tt, args.vspec) + coff;
            if constexpr (W == 16) {
                // quad layout: v[8m + 2i + h] = half h of rows 16m + 4k4 ..
                // 16m + 4k4 + 3 of tile column 32 warp + q4 + 8i
                const float2 *pq = args.psi + insert_zeros(tt, args.vspec) + coffq + 4 * k4;
#pragma unroll
                for (int m = 0; m < Sh::kRows / 16; ++m)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        ld_v8(pq + args.qoff[i] + args.rdep[16 * m], v[8 * m + 2 * i], v[8 * m + 2 * i + 1]);
            } else if constexpr (W == 4) {
#pragma unroll
                for (int j = 0; j < Sh::kRows / 4; ++j) ld_v8(p + args.rdep[4 * j], v[2 * j], v[2 * j + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < Sh::kRows / 2; ++j) {
                    if constexpr (W == 2) {
                        v[j] = *(const float4 *)(p + args.rdep[2 * j]);
                    } else {
                        const float2 a = p[args.rdep[2 * j]], b = p[args.rdep[2 * j + 1]];
                        v[j] = make_float4(a.x, a.y, b.x, b.y);
                    }
                }
            }
        };
        auto epilogue = [&](uint64_t tt) {
            float2 *const pb = args.psi + insert_zeros(tt, args.vspec);
            float2 *p = pb + coff;
            // four FP32 partial sums (chains of 2^K / 2 terms): the rounding
            // of a long chain is systematic when many amplitudes are equal;
            // FP64 across tiles (an FP64 add per 16 rows measured 1.2 %
            // slower)
            float ssq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int chunk = 0; chunk < Sh::kN / 32; ++chunk) {
                if constexpr (W == 16) {
                    // output rows 16 chunk + 4k4 .. + 3 of tile columns
                    // 32 warp + q4 + 8i: 32-byte stores, four lanes per line
                    float2 *pq = pb + coffq + 4 * k4 + args.rdep[16 * chunk];
#pragma unroll
                    for (int b2 = 0; b2 < 2; ++b2) {
                        float d[16];  // d[4 rho + 2c + a]: row 16 chunk + 4k4 + rho of column i = 2 b2 + c
                        tmem_ld16x256b_x4(lanes + ((uint32_t)(16 * b2) << 16) + Sh::kColD + chunk * 32, d);
#pragma unroll
                        for (int q = 0; q < 16; ++q) ssq[q & 3] = fmaf(d[q], d[q], ssq[q & 3]);
#pragma unroll
                        for (int c = 0; c < 2; ++c)
                            st_v8(pq + args.qoff[2 * b2 + c],
                                  make_float4(d[2 * c] * scale, d[2 * c + 1] * scale, d[4 + 2 * c] * scale,
                                              d[5 + 2 * c] * scale),
                                  make_float4(d[8 + 2 * c] * scale, d[9 + 2 * c] * scale, d[12 + 2 * c] * scale,
                                              d[13 + 2 * c] * scale));
                    }
                } else {
                float d[32];  // rows 16 chunk .. 16 chunk + 15, (re, im) interleaved
                tmem_ld32(lanes + Sh::kColD + chunk * 32, d);
#pragma unroll
                for (int q = 0; q < 32; ++q) ssq[q & 3] = fmaf(d[q], d[q], ssq[q & 3]);
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const int r = chunk * 16 + q;
                    const float4 o = make_float4(d[2 * q] * scale, d[2 * q + 1] * scale, d[2 * q + 2] * scale,
                                                 d[2 * q + 3] * scale);
                    if constexpr (W == 4) {
                        if (q % 4 == 0) {
                            const float4 o2 = make_float4(d[2 * q + 4] * scale, d[2 * q + 5] * scale,
                                                          d[2 * q + 6] * scale, d[2 * q + 7] * scale);
                            st_v8(p + args.rdep[r], o, o2);
                        }
                    } else if constexpr (W == 2) {
                        *(float4 *)(p + args.rdep[r]) = o;
                    } else {
                        p[args.rdep[r]] = make_float2(o.x, o.y);
                        p[args.rdep[r + 1]] = make_float2(o.z, o.w);
                    }
                }
                }
            }
            nrm_out += (double)((ssq[0] + ssq[1]) + (ssq[2] + ssq[3]));
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
            float xsq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int chunk = 0; chunk < Sh::kRows / 16; ++chunk) {
                if constexpr (W == 16) {
                    // lanes 32 warp + 16 b2 + q4 + 8c (tile column i = 2 b2 + c),
                    // A columns 16 chunk + 8h + 2k4 + e = rows 16 chunk + 4k4 + 2h + e
#pragma unroll
                    for (int b2 = 0; b2 < 2; ++b2) {
                        uint32_t hw[8], lw[8];
#pragma unroll
                        for (int c = 0; c < 2; ++c)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float4 x = v[8 * chunk + 2 * (2 * b2 + c) + h];
                                xsq[0] = fmaf(x.x, x.x, xsq[0]);
                                xsq[1] = fmaf(x.y, x.y, xsq[1]);
                                xsq[2] = fmaf(x.z, x.z, xsq[2]);
                                xsq[3] = fmaf(x.w, x.w, xsq[3]);
                                split_pair(x.x, x.y, hw[4 * h + 2 * c], lw[4 * h + 2 * c]);
                                split_pair(x.z, x.w, hw[4 * h + 2 * c + 1], lw[4 * h + 2 * c + 1]);
                            }
                        const uint32_t l16 = lanes + ((uint32_t)(16 * b2) << 16) + chunk * 16;
                        tmem_st16x256b_x2(l16 + Sh::kColAHi, hw);
                        tmem_st16x256b_x2(l16 + Sh::kColALo, lw);
                    }
                } else {
                    // this lane's own column: A columns 16 chunk + j = rows
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 x = v[chunk * 8 + j];
                        xsq[0] = fmaf(x.x, x.x, xsq[0]);
                        xsq[1] = fmaf(x.y, x.y, xsq[1]);
                        xsq[2] = fmaf(x.z, x.z, xsq[2]);
                        xsq[3] = fmaf(x.w, x.w, xsq[3]);
                        split_pair(x.x, x.y, hw[2 * j], lw[2 * j]);
                        split_pair(x.z, x.w, hw[2 * j + 1], lw[2 * j + 1]);
                    }
                    tmem_st16(lanes + Sh::kColAHi + chunk * 16, hw);
                    tmem_st16(lanes + Sh::kColALo + chunk * 16, lw);
                }
            }
            nrm_in += (double)((xsq[0] + xsq[1]) + (xsq[2] + xsq[3]));
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
                    // (A part, B part): X1R1, X2R1, X1R2, X2R2, X1R3.  (Issuing
                    // the small products first measured a 3x larger coherent
                    // error on Grover's search, the same on random circuits.)
                    const uint32_t a = tmem + ((term == 1 || term == 3) ? Sh::kColALo : Sh::kColAHi);
                    const uint32_t b = b0 + (uint32_t)(term < 2 ? 0 : (term < 4 ? 1 : 2)) * Sh::kBPart;
#pragma unroll
                    for (int kk = 0; kk < Sh::kN / 16; ++kk) {
                        mma_ts(tmem + Sh::kColD, a + kk * 8, sw128_desc(b + (kk >> 2) * Sh::kBHalf + (kk & 3) * 32),
                               Sh::kIdesc, acc);
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
    if (tid == 0)
        qsim_chain::chain_sums(args.chain, s_red[0] + s_red[2] + s_red[4] + s_red[6],
                               s_red[1] + s_red[3] + s_red[5] + s_red[7]);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::kCols) : "memory");
    }
}

// The B operand image: the nsplit bf16 parts of R = real form of U (D = 2^K
// rows), each N rows (output index 2j+a) x N K elements (input index 2j'+b)
// in K halves of 64 elements; within a half, row `row` is 128 bytes at
// row * 128 with its 16-byte chunks XOR-swizzled by row & 7.  Output j is
// block row orow(j) and input j' block row irow(j'): the identity, or for
// the quad fragments of W = 16 (see k_block_tmem) orow(16G + 4h + k) =
// 16G + 4k + h and irow(16G + 8h + 2k + e) = 16G + 4k + 2h + e.
int quad_out_row(int j) { return (j & ~15) | ((j & 3) << 2) | ((j >> 2) & 3); }
int quad_in_row(int j) { return (j & ~15) | (((j >> 1) & 3) << 2) | (((j >> 3) & 1) << 1) | (j & 1); }

void build_operand(const cd *U, int K, int nsplit, bool quad, std::vector<unsigned char> &rec) {
    const int D = 1 << K, N = 2 * D, half = N * 128, part = (N / 64) * half;
    rec.assign((size_t)nsplit * part, 0);
    for (int row = 0; row < N; ++row)
        for (int k = 0; k < N; ++k) {
            const int ro = quad ? quad_out_row(row >> 1) : row >> 1;
            const int ri = quad ? quad_in_row(k >> 1) : k >> 1;
            const cd u = U[ro * D + ri];
            const int a = row & 1, b = k & 1;
            double rem = a == 0 ? (b == 0 ? u.real() : -u.imag()) : (b == 0 ? u.imag() : u.real());
            const int kb = (k & 63) * 2;
            const size_t off =
                (size_t)(k >> 6) * half + (size_t)row * 128 + ((((kb >> 4) ^ (row & 7)) << 4)) + (kb & 15);
            for (int sp = 0; sp < nsplit; ++sp) {
                const uint16_t h = f32_to_bf16_bits((float)rem);
                rem -= bf16_bits_to_double(h);
                std::memcpy(&rec[(size_t)sp * part + off], &h, 2);
            }
        }
}

template <int K>
int launch_tmem(qsim *s, const int *qubits, const cd *m) {
    using Sh = TmShape<K>;
    const int n = s->n;
    const int nsplit = s->tc_terms == 5 ? 3 : 2;
    TmArgs a{};
    uint64_t Smask = 0;
    for (int j = 0; j < K; ++j) Smask |= 1ull << qubits[j];
    uint64_t Vmask = Smask;
    for (int b = 0, nf = 0; b < n && nf < 7; ++b)
        if (!((Smask >> b) & 1ull)) {
            a.fpos[nf++] = b;
            Vmask |= 1ull << b;
        }
    a.vspec.m = Sh::kTileBits;
    for (int b = 0, k = 0; b < n; ++b)
        if ((Vmask >> b) & 1ull) a.vspec.pos[k++] = b;
    for (int r = 0; r < Sh::kRows; ++r) {
        uint64_t d = 0;
        for (int j = 0; j < K; ++j)
            if ((r >> j) & 1) d |= 1ull << qubits[j];
        a.rdep[r] = d;
    }
    // W = 16: tile columns 32w + q + 8i lie qoff[i] from 32w + q
    for (int i = 0; i < 4; ++i)
        a.qoff[i] = ((i & 1) ? 1ull << a.fpos[3] : 0ull) + ((i & 2) ? 1ull << a.fpos[4] : 0ull);
    // amplitudes per global access (see k_block_tmem)
    const bool low4 = qubits[0] == 0 && qubits[1] == 1 && qubits[2] == 2 && qubits[3] == 3;
    const int W = low4 ? 16 : (qubits[0] == 0 && qubits[1] == 1) ? 4 : (qubits[0] == 0 ? 2 : 1);
    const int wi = W == 16 ? 3 : W == 4 ? 2 : W - 1;

    std::vector<unsigned char> rec;
    build_operand(m, K, nsplit, W == 16, rec);
    unsigned char *dev_rec = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev_rec);
    if (rc) return rc;

    auto kernel = W == 16 ? k_block_tmem<K, 16>
                          : W == 4 ? k_block_tmem<K, 4> : (W == 2 ? k_block_tmem<K, 2> : k_block_tmem<K, 1>);
    const int dev = s->device;
    if (dev < 0 || dev >= 64) return QSIM_ENOTSUP;
    static int smem_for[4][64][4] = {{{0}}};  // [access width][device][nsplit]: dynamic shared memory to request
    static int smem_attr[4][64] = {{0}};      // [access width][device]: the kernel's shared-memory limit set so far
    int &smem = smem_for[wi][dev][nsplit];
    if (!smem) {
        // At most kCtasPerSm CTAs per SM, as many as the tensor memory holds
        // (512 columns).  If registers and shared memory would let another
        // CTA in, request more shared memory so that it stays out: its
        // allocation would wait for one of the others to finish and
        // unbalance the persistent grid.
        cudaFuncAttributes fa;
        int regs_sm = 65536, smem_sm = 233472;
        cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return cuda_err(s, e, "tmem block kernel attributes");
        int bytes = 1024 + nsplit * Sh::kBPart + kTmExtra;
        const int cap = Sh::kCtasPerSm;
        const int by_regs = regs_sm / (fa.numRegs * kTmThreads);
        if (by_regs > cap && smem_sm / (bytes + 1024) > cap) bytes = smem_sm / (cap + 1) - 1024 + 64;
        // the limit is per kernel, shared by both operand sizes: only raise it
        if (bytes > smem_attr[wi][dev]) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return cuda_err(s, e, "tmem block kernel attribute");
            smem_attr[wi][dev] = bytes;
        }
        if (getenv("QSIM_DEBUG"))
            fprintf(stderr, "qsim: k_block_tmem<%d,%d> regs %d smem %d (registers allow %d CTAs/SM, cap %d)\n", K, W,
                    fa.numRegs, bytes, by_regs, cap);
        smem = bytes;
    }
    a.psi = (float2 *)s->state;
    a.rec = dev_rec;
    a.rec_bytes = (uint32_t)rec.size();
    a.nsplit = nsplit;
    a.ntiles = 1ull << (n - Sh::kTileBits);
    a.err = (unsigned int *)((char *)s->ws + kWsErr);
    uint64_t cap = (uint64_t)s->sms * Sh::kCtasPerSm;
    if (cap > (uint64_t)kMaxTcGrid) cap = kMaxTcGrid;
    const uint64_t grid = a.ntiles < cap ? a.ntiles : cap;
    a.chain = qsim_chain::chain_next(s);
    kernel<<<(unsigned)grid, kTmThreads, smem, s->stream>>>(a);
    s->stats.launches++;
    qsim_chain::chain_advance(s, (int)grid);
    return cuda_err(s, cudaGetLastError(), "tmem block launch");
}

// Embed a k-qubit block (k < 5) into the 5-qubit block on its qubits and the
// lowest qubits outside them (identity on the added ones), so that it runs
// on the 5-qubit kernel.  q5 receives the 5 qubits in ascending order.
void pad_to_five(int n, const int *q, int k, const cd *m, int *q5, std::vector<cd> &m5) {
    uint64_t S = 0;
    for (int j = 0; j < k; ++j) S |= 1ull << q[j];
    uint64_t S5 = S;
    for (int b = 0; b < n && __builtin_popcountll(S5) < 5; ++b) S5 |= 1ull << b;
    int kk = 0;
    for (int b = 0; b < n; ++b)
        if ((S5 >> b) & 1ull) q5[kk++] = b;
    int pos[5] = {0, 0, 0, 0, 0};  // position in q5 of block qubit j
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < 5; ++i)
            if (q5[i] == q[j]) pos[j] = i;
    uint32_t added = 0;  // positions (in q5) of the added qubits
    for (int i = 0; i < 5; ++i)
        if (!((S >> q5[i]) & 1ull)) added |= 1u << i;
    const int D = 1 << k;
    m5.assign(32 * 32, cd(0.0, 0.0));
    for (int r = 0; r < 32; ++r)
        for (int c = 0; c < 32; ++c) {
            if ((r & added) != (c & added)) continue;
            int ro = 0, co = 0;
            for (int j = 0; j < k; ++j) {
                ro |= ((r >> pos[j]) & 1) << j;
                co |= ((c >> pos[j]) & 1) << j;
            }
            m5[r * 32 + c] = m[ro * D + co];
        }
}

}  // namespace

int launch_block_tmem(qsim *s, const int *qubits, int k, const cd *m) {
    if (s->prec != QSIM_C64 || !s->tc_enabled || (k != 5 && k != 6) || s->n < k + 7) return QSIM_ENOTSUP;
    return k == 6 ? launch_tmem<6>(s, qubits, m) : launch_tmem<5>(s, qubits, m);
}

int launch_block_tc(qsim *s, const int *qubits, int k, const cd *m) {
    if (s->prec != QSIM_C64 || !s->tc_enabled || k < 4 || k > 5 || s->n < 12) return QSIM_ENOTSUP;
    if (k == 5) return launch_tmem<5>(s, qubits, m);
    int q5[5];
    std::vector<cd> m5;
    pad_to_five(s->n, qubits, k, m, q5, m5);
    return launch_tmem<5>(s, q5, m5.data());
}

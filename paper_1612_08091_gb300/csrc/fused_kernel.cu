// fused_kernel.cu -- a fused 5-qubit block applied on the tensor cores
// (tcgen05 / TMEM), complex64 amplitudes, BF16x3 split products.
//
// The paper's simulator gains its speed from lazily buffering gates and
// executing them together (ProjectQ paper, Sec. 4.3.2, Fig. 7 caption).
// Here a run of gates on at most 5 qubits S = {s0 < ... < s4} has been
// multiplied into one 32 x 32 complex matrix U.  Viewing the state as a
// 32 x 2^(n-5) matrix Psi (row r = the bits of S, column = the other bits),
// the pass computes Psi' = U Psi.
//
// Real form.  With interleaved (re, im) amplitudes, the 64-wide real vector
// x of one column (x[2r] = Re psi_r, x[2r+1] = Im psi_r) maps to y = R x
// with R[2r+a][2r'+b] the 2x2 real block of U[r][r'].  A tile of 128 columns
// is the GEMM  D(128 x 64) = X(128 x 64) R^T(64 x 64),  M = 128 (columns),
// N = 64 (outputs), K = 64 (inputs): operand A = X (state, K-major), operand
// B = R (gate, K-major, i.e. R itself row by row), D in tensor memory.
//
// BF16x3.  X = X1 + X2 and R = R1 + R2 (+ R3) are split into bfloat16
// parts (X2 = bf16(X - X1), ...); the products X1 R1 + X2 R1 + X1 R2 (three
// terms, or five with X2 R2 + X1 R3) accumulate in FP32 in tensor memory.
// The state split loses about 2^-16 relatively per pass (incoherently); the
// gate split is pre-computed on the host in FP64.
//
// Tiles.  The tile's 128 columns take the 7 lowest qubits F outside S, so a
// tile is the 2^12 amplitudes whose index bits outside V = S u F are fixed;
// V always contains qubits 0..6 (or more), so every tile is made of runs of
// at least 128 contiguous amplitudes.
//
// Per CTA (persistent, 128 threads, two CTAs per SM):
//   - one TMA bulk copy brings the gate operand R1, R2(, R3) (pre-swizzled
//     on the host) and the tile index tables into shared memory;
//   - each thread loads 32 amplitudes of the next tile with 16-byte loads,
//     splits them into bf16 hi/lo and writes them to the A buffers in the
//     128-byte-swizzled K-major layout the MMA reads;
//   - thread 0 issues 12 (or 20) tcgen05.mma (M128 N64 K16) into one of two
//     TMEM accumulators and commits them to an mbarrier;
//   - while the tensor cores work and the next tile's loads are in flight,
//     the four warps read the previous tile's accumulator with tcgen05.ld
//     (warp w owns TMEM lanes 32w..32w+31 = tile columns) and store it.
// Every wait is bounded; on time-out the kernel raises an error flag in the
// workspace, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kTcThreads = 128;
constexpr int kTile = 4096;              // amplitudes per tile (2^12)
constexpr int kABytes = 128 * 128;       // one bf16 split of X: 128 rows x 128 B
constexpr int kBBytes = 64 * 128;        // one bf16 split of R: 64 rows x 128 B
constexpr int kTablesBytes = 2560;
constexpr uint32_t kTmemCols = 128;      // two 64-column fp32 accumulators
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kMaxTcGrid = 2 * kSMs;

// Layout of the per-block operand record (host-built, copied to smem as is).
struct RecTables {
    uint64_t t_lo[64];   // address bits of tile element e (low 6 bits of e)
    uint64_t t_hi[64];   // ... (high 6 bits of e)
    uint64_t cdep[128];  // address bits of tile column c
    uint64_t rdep[32];   // address bits of block row r
    uint8_t r_lo[64], r_hi[64];  // block row of element e
    uint8_t c_lo[64], c_hi[64];  // tile column of element e
};
static_assert(sizeof(RecTables) == kTablesBytes, "table layout");

struct TcArgs {
    float2 *psi;
    const unsigned char *rec;  // operand record in global memory (16-B aligned)
    uint32_t rec_bytes;
    int nsplit;                // bf16 parts of R: 2 (BF16x3) or 3 (five products)
    uint64_t ntiles;
    InsertSpec vspec;          // the 12 positions of V, ascending
    unsigned int *err;         // error flag
    // norm tracking: this pass writes per-CTA sums of |x|^2 (inputs) and
    // |y|^2 (raw outputs) to norm_out[0..grid) and [kMaxTcGrid..); the
    // previous pass's sums (norm_prev, prev_grid CTAs, or null) give the
    // output scale sqrt(in/out)
    double *norm_out;
    const double *norm_prev;
    int prev_grid;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 64-bit shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of
// 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor: D fp32, A and B bf16, both K-major, M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_half, float hi_half) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo_half, hi_half);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// Write one amplitude (re, im) at block row r of tile column c into the hi
// and lo A buffers (128-byte swizzle: 16-byte chunk index ^= row & 7).
__device__ __forceinline__ void put_amp(unsigned char *a_hi, unsigned char *a_lo, int c, int r, float re, float im) {
    const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi_ = __float2bfloat16_rn(im);
    const float rr = re - __bfloat162float(hr), ri = im - __bfloat162float(hi_);
    __nv_bfloat162 h2;
    h2.x = hr;
    h2.y = hi_;
    uint32_t hw;
    memcpy(&hw, &h2, 4);
    const uint32_t lw = pack_bf16x2(rr, ri);
    const int off = c * 128 + ((((r >> 2) ^ c) & 7) << 4) + ((r & 3) << 2);
    *(uint32_t *)(a_hi + off) = hw;
    *(uint32_t *)(a_lo + off) = lw;
}

__global__ void __launch_bounds__(kTcThreads, 2) k_block_tc(const TcArgs args) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *A = smem;                           // [2 buf][2 split][kABytes]
    unsigned char *B = smem + 4 * kABytes;             // [nsplit][kBBytes] then tables
    const RecTables *tab = (const RecTables *)(B + args.nsplit * kBBytes);
    uint64_t *bars = (uint64_t *)(B + args.nsplit * kBBytes + kTablesBytes);  // [0]=operand, [1],[2]=mma
    uint32_t *tmem_slot = (uint32_t *)(bars + 3);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *s_scale = (float *)(tmem_slot + 2);
    double *s_red = (double *)(bars + 5);  // [4 warps][2]

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        *abort_flag = 0;
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
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[0])),
                     "r"(args.rec_bytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(B)),
                     "l"(args.rec), "r"(args.rec_bytes), "r"(smem_u32(&bars[0]))
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    bool ok = mbar_wait(&bars[0], 0);
    if (!ok) {
        atomicOr(args.err, 1u);
        *abort_flag = 1;
    }
    __syncthreads();

    const float2 *psi_in = args.psi;
    float2 *psi = args.psi;
    double nrm_in = 0.0, nrm_out = 0.0;
    const float scale = *s_scale;
    if (!*abort_flag) {
        // per-thread constants of the element mapping e = 2*(tid + 128 i) + h
        const int elo0 = (2 * tid) & 63, elo1 = (2 * tid + 1) & 63;
        const uint64_t toff_lo = tab->t_lo[elo0];
        const int rl0 = tab->r_lo[elo0], rl1 = tab->r_lo[elo1];
        const int cl0 = tab->c_lo[elo0], cl1 = tab->c_lo[elo1];
        const int ehi0 = tid >> 5;
        const uint64_t my_cdep = tab->cdep[tid];
        const int nterms = args.nsplit == 3 ? 5 : 3;

        float4 regs[16];
        uint64_t t = blockIdx.x;
        auto load_tile = [&](uint64_t tt) {
            const uint64_t base = insert_zeros(tt, args.vspec);
            const float2 *p = psi_in + base + toff_lo;
#pragma unroll
            for (int i = 0; i < 16; ++i) regs[i] = *(const float4 *)(p + tab->t_hi[ehi0 + 4 * i]);
        };
        auto epilogue = [&](uint64_t tt, int j) {
            const int buf = j & 1;
            if (!mbar_wait(&bars[1 + buf], (uint32_t)((j >> 1) & 1))) {
                atomicOr(args.err, 2u);
                *abort_flag = 1;
                return;
            }
            tc_fence_after();
            const uint64_t base = insert_zeros(tt, args.vspec) + my_cdep;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * 64);
            float ssq = 0.f;
#pragma unroll
            for (int chunk = 0; chunk < 4; ++chunk) {
                float v[16];
                tmem_ld16(taddr + chunk * 16, v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int r = chunk * 8 + q;
                    ssq = fmaf(v[2 * q], v[2 * q], fmaf(v[2 * q + 1], v[2 * q + 1], ssq));
                    psi[base + tab->rdep[r]] = make_float2(v[2 * q] * scale, v[2 * q + 1] * scale);
                }
            }
            nrm_out += (double)ssq;
            tc_fence_before();
        };

        if (t < args.ntiles) load_tile(t);
        int it = 0;
        for (; t < args.ntiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            unsigned char *a_hi = A + (2 * buf) * kABytes;
            unsigned char *a_lo = A + (2 * buf + 1) * kABytes;
            float xsq = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                xsq = fmaf(regs[i].x, regs[i].x, fmaf(regs[i].y, regs[i].y, xsq));
                xsq = fmaf(regs[i].z, regs[i].z, fmaf(regs[i].w, regs[i].w, xsq));
                const int eh = ehi0 + 4 * i;
                const int rh = tab->r_hi[eh], ch = tab->c_hi[eh];
                put_amp(a_hi, a_lo, cl0 | ch, rl0 | rh, regs[i].x, regs[i].y);
                put_amp(a_hi, a_lo, cl1 | ch, rl1 | rh, regs[i].z, regs[i].w);
            }
            nrm_in += (double)xsq;
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (*abort_flag) break;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * 64);
                const uint32_t ahi = smem_u32(a_hi), alo = smem_u32(a_lo);
                const uint32_t b0 = smem_u32(B), b1 = b0 + kBBytes, b2 = b0 + 2 * kBBytes;
                uint32_t acc = 0;
                for (int term = 0; term < nterms; ++term) {
                    // (A part, B part): X1R1, X2R1, X1R2, X2R2, X1R3
                    const uint32_t a = (term == 1 || term == 3) ? alo : ahi;
                    const uint32_t b = term < 2 ? b0 : (term < 4 ? b1 : b2);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        mma_bf16(d, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), acc);
                        acc = 1;
                    }
                }
                mma_commit(&bars[1 + buf]);
            }
            const uint64_t tn = t + gridDim.x;
            if (tn < args.ntiles) load_tile(tn);
            if (it >= 1) epilogue(t - gridDim.x, it - 1);
        }
        if (it >= 1 && !*abort_flag) epilogue(t - gridDim.x, it - 1);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
uint16_t f32_to_bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t round = 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)((u + round) >> 16);
}
double bf16_bits_to_double(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

// Embed a k-qubit block (k < 5) into 5 qubits by adding the lowest qubits
// not in S, on which it acts as the identity.
void pad_to_five(int n, const int *q, int k, const cd *m, int *q5, std::vector<cd> &m5) {
    uint64_t S = 0;
    for (int j = 0; j < k; ++j) S |= 1ull << q[j];
    uint64_t S5 = S;
    for (int b = 0; b < n && __builtin_popcountll(S5) < 5; ++b) S5 |= 1ull << b;
    int pos_old[5];
    int kk = 0;
    for (int b = 0; b < n; ++b)
        if ((S5 >> b) & 1ull) q5[kk++] = b;
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < 5; ++i)
            if (q5[i] == q[j]) pos_old[j] = i;
    uint32_t newmask = 0;  // positions (in 5) of added qubits
    for (int i = 0; i < 5; ++i)
        if (!((S >> q5[i]) & 1ull)) newmask |= 1u << i;
    const int D = 1 << k;
    m5.assign(32 * 32, cd(0.0, 0.0));
    for (int r = 0; r < 32; ++r)
        for (int c = 0; c < 32; ++c) {
            if ((r & newmask) != (c & newmask)) continue;
            int ro = 0, co = 0;
            for (int j = 0; j < k; ++j) {
                ro |= ((r >> pos_old[j]) & 1) << j;
                co |= ((c >> pos_old[j]) & 1) << j;
            }
            m5[r * 32 + c] = m[ro * D + co];
        }
}

void build_record(int n, const int *S, const cd *U, int nsplit, std::vector<unsigned char> &rec, InsertSpec &vspec) {
    // R[2r+a][2r'+b]: real 2x2 block of U[r][r']
    double R[64][64];
    for (int r = 0; r < 32; ++r)
        for (int c = 0; c < 32; ++c) {
            const double ur = U[r * 32 + c].real(), ui = U[r * 32 + c].imag();
            R[2 * r][2 * c] = ur;
            R[2 * r][2 * c + 1] = -ui;
            R[2 * r + 1][2 * c] = ui;
            R[2 * r + 1][2 * c + 1] = ur;
        }
    rec.assign((size_t)nsplit * kBBytes + kTablesBytes, 0);
    for (int row = 0; row < 64; ++row)
        for (int k = 0; k < 64; ++k) {
            double rem = R[row][k];
            for (int sp = 0; sp < nsplit; ++sp) {
                const uint16_t h = f32_to_bf16_bits((float)rem);
                rem -= bf16_bits_to_double(h);
                const int off = row * 128 + ((((k * 2) >> 4) ^ (row & 7)) << 4) + ((k * 2) & 15);
                std::memcpy(&rec[(size_t)sp * kBBytes + off], &h, 2);
            }
        }
    // V = S u F, F = lowest 7 qubits outside S
    uint64_t Smask = 0;
    for (int j = 0; j < 5; ++j) Smask |= 1ull << S[j];
    int F[7], nf = 0;
    for (int b = 0; b < n && nf < 7; ++b)
        if (!((Smask >> b) & 1ull)) F[nf++] = b;
    const uint64_t Vmask = Smask | [&] {
        uint64_t m = 0;
        for (int j = 0; j < 7; ++j) m |= 1ull << F[j];
        return m;
    }();
    int V[12], nv = 0;
    for (int b = 0; b < n; ++b)
        if ((Vmask >> b) & 1ull) V[nv++] = b;
    vspec = InsertSpec{};
    vspec.m = 12;
    for (int j = 0; j < 12; ++j) vspec.pos[j] = V[j];
    RecTables T;
    std::memset(&T, 0, sizeof(T));
    auto s_index = [&](int bit) {
        for (int j = 0; j < 5; ++j)
            if (S[j] == bit) return j;
        return -1;
    };
    auto f_index = [&](int bit) {
        for (int j = 0; j < 7; ++j)
            if (F[j] == bit) return j;
        return -1;
    };
    for (int e = 0; e < 64; ++e) {
        for (int half = 0; half < 2; ++half) {
            uint64_t addr = 0;
            int r = 0, c = 0;
            for (int b = 0; b < 6; ++b) {
                if (!((e >> b) & 1)) continue;
                const int bit = V[6 * half + b];
                addr |= 1ull << bit;
                const int si = s_index(bit);
                if (si >= 0)
                    r |= 1 << si;
                else
                    c |= 1 << f_index(bit);
            }
            if (half == 0) {
                T.t_lo[e] = addr;
                T.r_lo[e] = (uint8_t)r;
                T.c_lo[e] = (uint8_t)c;
            } else {
                T.t_hi[e] = addr;
                T.r_hi[e] = (uint8_t)r;
                T.c_hi[e] = (uint8_t)c;
            }
        }
    }
    for (int c = 0; c < 128; ++c) {
        uint64_t a = 0;
        for (int j = 0; j < 7; ++j)
            if ((c >> j) & 1) a |= 1ull << F[j];
        T.cdep[c] = a;
    }
    for (int r = 0; r < 32; ++r) {
        uint64_t a = 0;
        for (int j = 0; j < 5; ++j)
            if ((r >> j) & 1) a |= 1ull << S[j];
        T.rdep[r] = a;
    }
    std::memcpy(&rec[(size_t)nsplit * kBBytes], &T, sizeof(T));
}

size_t smem_bytes(int nsplit) { return 1024 + 4 * kABytes + (size_t)nsplit * kBBytes + kTablesBytes + 128; }

}  // namespace

int launch_block_tc(qsim *s, const int *qubits, int k, const cd *m) {
    if (s->prec != QSIM_C64 || s->n < 12 || k < 1 || k > 5) return QSIM_ENOTSUP;
    if (!s->tc_enabled) return QSIM_ENOTSUP;
    int q5[5];
    std::vector<cd> m5;
    const cd *U = m;
    if (k < 5) {
        pad_to_five(s->n, qubits, k, m, q5, m5);
        U = m5.data();
    } else {
        for (int j = 0; j < 5; ++j) q5[j] = qubits[j];
    }
    const int nsplit = s->tc_terms == 5 ? 3 : 2;
    std::vector<unsigned char> rec;
    TcArgs a{};
    build_record(s->n, q5, U, nsplit, rec, a.vspec);
    unsigned char *dev_rec = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev_rec);
    if (rc) return rc;
    static bool attr_set[64] = {false};
    const int dev = s->device;
    const size_t smem = smem_bytes(3);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_err(s, e, "tc kernel attribute");
        attr_set[dev] = true;
    }
    a.psi = (float2 *)s->state;
    a.rec = dev_rec;
    a.rec_bytes = (uint32_t)rec.size();
    a.nsplit = nsplit;
    a.ntiles = 1ull << (s->n - 12);
    a.err = (unsigned int *)((char *)s->ws + kWsErr);
    const uint64_t grid = a.ntiles < (uint64_t)kMaxTcGrid ? a.ntiles : (uint64_t)kMaxTcGrid;
    double *slots = (double *)((char *)s->ws + kWsNorm);
    const int slot = (int)(s->tc_passes & 1);
    a.norm_out = slots + slot * 2 * kMaxTcGrid;
    a.norm_prev = (s->norm_tracking && s->tc_passes > 0) ? slots + (slot ^ 1) * 2 * kMaxTcGrid : nullptr;
    a.prev_grid = s->tc_prev_grid;
    k_block_tc<<<(unsigned)grid, kTcThreads, smem, s->stream>>>(a);
    s->stats.launches++;
    s->tc_passes++;
    s->tc_prev_grid = (int)grid;
    return cuda_err(s, cudaGetLastError(), "tc block launch");
}

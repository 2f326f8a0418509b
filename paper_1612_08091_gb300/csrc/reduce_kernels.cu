// reduce_kernels.cu -- probabilities, collapse, full-register sampling and
// Pauli-sum expectation values.
//
// Measurement in the computational basis with collapse of the register is
// the paper's Measure operation (ProjectQ paper, Sec. 4 listing 1; Appendix
// A.1 teleportation; Appendix A.3 measure-and-reset).  The sums behind it
// are accumulated in FP64 where it carries precision: partial sums of
// |psi_i|^2 are formed in the amplitude precision over short runs (8 to 32
// terms for complex64, or a 1024-term tile reduced as a 5-level warp tree),
// then added in FP64 and reduced across blocks by a fixed-order second stage,
// so every result is deterministic for a given launch configuration.  FP64
// arithmetic runs at about 1/58 of the FP32 rate on this part, so one FP64
// add per amplitude would bound these passes below half the HBM bandwidth;
// the complex64 relative error stays below about 3e-6.
//
// Expectation values <psi|P|psi> of Pauli strings P (Z-only strings in one
// pass for all terms; strings with an X/Y part grouped by their X mask, one
// pass per group) use  P|i> = i^{#Y} (-1)^{popc(i & zmask)} |i ^ xmask>.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kRedThreads = 256;

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// all single-qubit probabilities in one pass
// ---------------------------------------------------------------------------
// A warp owns tiles of 1024 consecutive amplitudes; lane l reads index
// tile*1024 + 32*j + l for j = 0..31 (each j is a coalesced 32-amplitude
// run).  Per lane it sums w_j = |psi|^2 over all j (S) and over the j with
// bit b set (Sb[b]).  Then P(q=1) gets: for q < 5 the lanes with bit q set,
// for 5 <= q < 10 the warp sum of Sb[q-5], for q >= 10 the whole tile if bit
// q of the tile index is set.  Lane q accumulates qubit q (and q+32).
template <typename Amp>
__global__ void __launch_bounds__(kRedThreads) k_probs_tiles(const Amp *__restrict__ psi, int n, uint64_t ntiles,
                                                             double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[kRedThreads / 32][2 * 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double accA = 0.0, accB = 0.0, accN = 0.0;
    R fA = 0, fB = 0, fN = 0;  // the last <= 16 tiles, in the amplitude precision
    int pending = 0;
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
        // warp sums in the amplitude precision (a tree of 5 levels over
        // the lanes' 32-term sums); lane q collects qubit q (and q + 32)
        const R T = warp_sum(S);
        R mine = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const R a = warp_sum(((lane >> q) & 1) ? S : (R)0);
            if (lane == q) mine = a;
        }
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const R a = warp_sum(Sb[b]);
            if (lane == 5 + b) mine = a;
        }
        const uint64_t base = tile << 10;
        if (lane >= 10 && lane < n && ((base >> lane) & 1ull)) mine = T;
        fA += mine;
        if (lane + 32 < n && ((base >> (lane + 32)) & 1ull)) fB += T;
        fN += T;
        if (++pending == 16) {  // FP64 beyond 16 tiles
            accA += (double)fA;
            accB += (double)fB;
            accN += (double)fN;
            fA = fB = fN = 0;
            pending = 0;
        }
    }
    accA += (double)fA;
    accB += (double)fB;
    accN += (double)fN;
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

// Small registers (n < 10): one block, one amplitude per thread per step.
template <typename Amp>
__global__ void k_probs_small(const Amp *__restrict__ psi, int n, double *__restrict__ out) {
    __shared__ double sh[32];
    const uint64_t N = 1ull << n;
    for (int v = 0; v <= n; ++v) {
        double acc = 0.0;
        for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) {
            const double w = (double)norm2(psi[i]);
            if (v == 0 || ((i >> (v - 1)) & 1ull)) acc += w;
        }
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) out[v] = acc;
    }
}

// Fixed-order second stage: out[v] = sum_b partials[b*V + v].
__global__ void k_finalize(const double *__restrict__ partials, int nblocks, int V, double *__restrict__ out) {
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partials[(size_t)b * V + v];
        out[v] = t;
    }
}

// ---------------------------------------------------------------------------
// masked sums:  sum over {i : (i & mask) == value} of |psi_i|^2
// ---------------------------------------------------------------------------
template <typename Amp>
__global__ void __launch_bounds__(kRedThreads) k_masked_sum(const Amp *__restrict__ psi, uint64_t ngroups,
                                                            const InsertSpec ins, uint64_t value,
                                                            double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    double acc = 0.0;
    R run = 0;  // up to 4 rounds in the amplitude precision, FP64 beyond
    int rounds = 0;
    for (; g < ngroups; g += 16 * stride) {
        // the 16 indices first, then 16 loads in flight per thread
        uint64_t idx[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) idx[r] = insert_zeros(g + (uint64_t)r * stride, ins) | value;
#pragma unroll
        for (int r = 0; r < 16; ++r)
            if (g + (uint64_t)r * stride < ngroups) run += norm2(psi[idx[r]]);
        if (++rounds == 4) {
            acc += (double)run;
            run = 0;
            rounds = 0;
        }
    }
    acc += (double)run;
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Both halves of one qubit: partials[2b] = sum over bit q = 0, [2b+1] = bit 1.
template <typename Amp>
__global__ void __launch_bounds__(kRedThreads) k_split_sum(const Amp *__restrict__ psi, uint64_t npairs, int q,
                                                           double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t bit = 1ull << q, lowmask = bit - 1ull;
    uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    double a0 = 0.0, a1 = 0.0;
    R r0 = 0, r1 = 0;  // up to 4 rounds in the amplitude precision, FP64 beyond
    int rounds = 0;
    for (; g < npairs; g += 8 * stride) {
        // 16 loads in flight per thread
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint64_t gr = g + (uint64_t)r * stride;
            if (gr < npairs) {
                const uint64_t i0 = ((gr & ~lowmask) << 1) | (gr & lowmask);
                r0 += norm2(psi[i0]);
                r1 += norm2(psi[i0 | bit]);
            }
        }
        if (++rounds == 4) {
            a0 += (double)r0;
            a1 += (double)r1;
            r0 = r1 = 0;
            rounds = 0;
        }
    }
    a0 += (double)r0;
    a1 += (double)r1;
    a0 = block_sum(a0, sh);
    a1 = block_sum(a1, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a0;
        partials[2 * blockIdx.x + 1] = a1;
    }
}

// ---------------------------------------------------------------------------
// one qubit's halves in tiles:  S0 = sum over bit q = 0, S1 = over bit q = 1
// ---------------------------------------------------------------------------
// Tiles of 1024 consecutive amplitudes as in k_probs_tiles (lane l reads
// index tile*1024 + 32*j + l): bit q of an element is a lane bit (q < 5), a
// run bit (q < 10) or a bit of the tile index.  With only_set and q >= 10,
// only the tiles with bit q set are read (tile t' of ntiles = 2^(n-11) gets a
// 1 inserted at bit q - 10): half the state.
template <typename Amp>
__global__ void __launch_bounds__(kRedThreads) k_bit_sums(const Amp *__restrict__ psi, int q, uint64_t ntiles,
                                                          int only_set, double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double a0 = 0.0, a1 = 0.0;
    R f0 = 0, f1 = 0;  // the last <= 16 tiles, in the amplitude precision
    int pending = 0;
    const int tq = q - 10;
    for (uint64_t t = (uint64_t)blockIdx.x * nw + warp; t < ntiles; t += (uint64_t)gridDim.x * nw) {
        uint64_t tile = t;
        if (only_set && tq >= 0) tile = ((t >> tq) << (tq + 1)) | (1ull << tq) | (t & ((1ull << tq) - 1ull));
        const Amp *p = psi + (tile << 10) + lane;
        R w[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = norm2(p[j * 32]);
        R s0 = 0, s1 = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int bit = q < 5 ? (lane >> q) & 1 : (q < 10 ? (j >> (q - 5)) & 1 : (int)((tile >> tq) & 1ull));
            if (bit)
                s1 += w[j];
            else
                s0 += w[j];
        }
        f0 += s0;
        f1 += s1;
        if (++pending == 16) {  // FP64 beyond 16 tiles
            a0 += (double)f0;
            a1 += (double)f1;
            f0 = f1 = 0;
            pending = 0;
        }
    }
    a0 += (double)f0;
    a1 += (double)f1;
    a0 = block_sum(a0, sh);
    a1 = block_sum(a1, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a0;
        partials[2 * blockIdx.x + 1] = a1;
    }
}

// ---------------------------------------------------------------------------
// collapse: keep {i : (i & mask) == value} scaled by 1/sqrt(p), zero the rest
// ---------------------------------------------------------------------------
// The FP64 scale is applied to complex64 as a two-float split
// (s = s_hi + s_lo), so the only rounding is the final one to storage.
__device__ __forceinline__ double2 scale_amp(double2 a, double s, float, float) {
    return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ float2 scale_amp(float2 a, double, float shi, float slo) {
    return make_float2(fmaf(a.x, shi, a.x * slo), fmaf(a.y, shi, a.y * slo));
}

// One qubit q kept at value b: amplitude pairs (2k, 2k+1) move as one
// 16-byte (complex64) or two 16-byte (complex128) accesses; a pair that is
// dropped entirely is written as zeros without being read.
__device__ __forceinline__ void ld_pair(const float2 *p, float2 &a, float2 &b) {
    const float4 v = *(const float4 *)p;
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void st_pair(float2 *p, float2 a, float2 b) { *(float4 *)p = make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ void ld_pair(const double2 *p, double2 &a, double2 &b) {
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void st_pair(double2 *p, double2 a, double2 b) {
    p[0] = a;
    p[1] = b;
}

template <typename Amp>
__global__ void k_collapse_bit(Amp *__restrict__ psi, uint64_t npairs, int q, int b, double s, float shi,
                               float slo) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    Amp zero;
    zero.x = 0;
    zero.y = 0;
    uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    // 4 pairs per thread per round: the kept ones' loads go out together
    for (; k < npairs; k += 4 * stride) {
        Amp v0[4], v1[4];
        bool keep[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t kr = k + (uint64_t)r * stride;
            const uint64_t i = 2 * kr;
            keep[r] = kr < npairs && (q == 0 || (int)((i >> q) & 1ull) == b);
            if (keep[r]) ld_pair(psi + i, v0[r], v1[r]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t kr = k + (uint64_t)r * stride;
            if (kr >= npairs) continue;
            const uint64_t i = 2 * kr;
            if (!keep[r]) {
                st_pair(psi + i, zero, zero);
            } else if (q == 0) {
                st_pair(psi + i, b ? zero : scale_amp(v0[r], s, shi, slo), b ? scale_amp(v1[r], s, shi, slo) : zero);
            } else {
                st_pair(psi + i, scale_amp(v0[r], s, shi, slo), scale_amp(v1[r], s, shi, slo));
            }
        }
    }
}

template <typename Amp>
__global__ void k_collapse_mask(Amp *__restrict__ psi, uint64_t N, uint64_t mask, uint64_t value, double s,
                                float shi, float slo) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    // 8 elements per thread per round: the kept ones' loads go out together
    for (; i + 7 * stride < N; i += 8 * stride) {
        Amp v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint64_t k = i + (uint64_t)r * stride;
            if ((k & mask) == value) v[r] = psi[k];
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint64_t k = i + (uint64_t)r * stride;
            Amp z;
            if ((k & mask) == value) {
                z = scale_amp(v[r], s, shi, slo);
            } else {
                z.x = 0;
                z.y = 0;
            }
            psi[k] = z;
        }
    }
    for (; i < N; i += stride) {
        if ((i & mask) == value) {
            psi[i] = scale_amp(psi[i], s, shi, slo);
        } else {
            Amp z;
            z.x = 0;
            z.y = 0;
            psi[i] = z;
        }
    }
}

// ---------------------------------------------------------------------------
// expectation of Z-only strings:  sum_i |psi_i|^2 f(i),
// f(i) = sum_k c_k (-1)^{popc(i & z_k)}
// ---------------------------------------------------------------------------
// A warp owns tiles of 1024 amplitudes as in k_probs_tiles.  With j the
// run index (bits 5..9) and l the lane (bits 0..4), each lane forms the
// Walsh-Hadamard transform W^(m) = sum_j w_j (-1)^{popc(j & m)} of its 32
// weights; a term then contributes c_k (-1)^{popc(l & zl_k)}
// (-1)^{popc(tile & zh_k)} W^(m_k) with zl_k, m_k, zh_k = bits 0..4, 5..9
// and 10.. of z_k.  W^ is kept per warp in shared memory.  Terms with the
// same (zl, m) form a group whose tile-dependent signs fold into one
// coefficient per tile, formed by one lane per group and broadcast by warp
// shuffles, so the lanes' work scales with the groups (11 for a
// nearest-neighbour ZZ chain), not with the terms.
// Coefficients come in both precisions so that the complex64 kernel does
// no FP64 arithmetic per term (FP64, conversions included, runs at 1/58 of
// the FP32 rate here); tile indices and zh fit 32 bits (n <= 36).
constexpr int kMaxZTerms = 96;
struct ZTerms {
    int nt, ng;
    double c[kMaxZTerms];   // terms, grouped: group g owns [first[g], first[g+1])
    float cf[kMaxZTerms];   // the same, rounded to float
    unsigned zh[kMaxZTerms];
    int first[kMaxZTerms + 1];
    int zl[kMaxZTerms], m[kMaxZTerms];
};
static_assert(sizeof(ZTerms) <= 4000, "kernel parameter size");

__device__ __forceinline__ float zcoef(const ZTerms &T, int k, float) { return T.cf[k]; }
__device__ __forceinline__ double zcoef(const ZTerms &T, int k, double) { return T.c[k]; }

constexpr int kZThreads = 128;

template <typename Amp>
__global__ void __launch_bounds__(kZThreads) k_expect_z_tiles(const Amp *__restrict__ psi, uint64_t ntiles,
                                                              const ZTerms T, double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ R wh[kZThreads / 32][32][32];
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double acc = 0.0;
    R facc = 0;  // the last <= 16 tiles, in the amplitude precision
    int pending = 0;
    for (uint64_t tile = (uint64_t)blockIdx.x * nw + warp; tile < ntiles; tile += (uint64_t)gridDim.x * nw) {
        const Amp *p = psi + (tile << 10) + lane;
        R w[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = norm2(p[j * 32]);
        // in-register Walsh-Hadamard transform over the 5 run bits
#pragma unroll
        for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if ((j & h) == 0) {
                    const R a = w[j], b = w[j + h];
                    w[j] = a + b;
                    w[j + h] = a - b;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 32; ++m) wh[warp][m][lane] = w[m];
        __syncwarp();
        R e = 0;
        const unsigned t32 = (unsigned)tile;
        for (int g0 = 0; g0 < T.ng; g0 += 32) {
            // lane j forms group g0 + j's coefficient for this tile; the
            // lanes then take the groups one by one from it
            R c = 0;
            if (g0 + lane < T.ng)
                for (int k = T.first[g0 + lane]; k < T.first[g0 + lane + 1]; ++k) {
                    const R ck = zcoef(T, k, R(0));
                    c += (__popc(t32 & T.zh[k]) & 1) ? -ck : ck;
                }
            const int gn = T.ng - g0 < 32 ? T.ng - g0 : 32;
            for (int j = 0; j < gn; ++j) {
                const R cj = __shfl_sync(0xffffffffu, c, j);
                const R v = wh[warp][T.m[g0 + j]][lane];
                e += (__popc(lane & T.zl[g0 + j]) & 1) ? -cj * v : cj * v;
            }
        }
        __syncwarp();
        facc += e;
        if (++pending == 16) {  // FP64 beyond 16 tiles
            acc += (double)facc;
            facc = 0;
            pending = 0;
        }
    }
    acc += (double)facc;
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename Amp>
__global__ void k_expect_z_small(const Amp *__restrict__ psi, uint64_t N, const ZTerms T, double *__restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = (double)norm2(psi[i]);
        double f = 0.0;
        for (int g = 0; g < T.ng; ++g)
            for (int k = T.first[g]; k < T.first[g + 1]; ++k) {
                const uint64_t z = (uint64_t)T.zl[g] | ((uint64_t)T.m[g] << 5) | ((uint64_t)T.zh[k] << 10);
                f += (__popcll(i & z) & 1) ? -T.c[k] : T.c[k];
            }
        acc += w * f;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = acc;
}

// ---------------------------------------------------------------------------
// expectation of strings sharing one X mask x != 0:
//   <psi|P|psi> = sum over pairs (i, j = i ^ x) with bit h of i clear
//                 of 2 Re[ i^{y} (-1)^{popc(i & z)} psi_i conj(psi_j) ]
// (h = highest bit of x, y = popc(x & z) = number of Y factors).
// ---------------------------------------------------------------------------
constexpr int kMaxXTerms = 32;
struct XTerms {
    int nt;
    uint64_t x;
    int h;
    double c[kMaxXTerms];
    uint64_t z[kMaxXTerms];
    int y4[kMaxXTerms];  // number of Y factors mod 4
};

template <typename Amp>
__global__ void __launch_bounds__(kRedThreads) k_expect_x(const Amp *__restrict__ psi, uint64_t npairs, const XTerms T,
                                                          double *__restrict__ partials) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t bit = 1ull << T.h, lowmask = bit - 1ull;
    double acc = 0.0;
    uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    while (g < npairs) {
        R run = 0;
#pragma unroll 1
        for (int r = 0; r < 8 && g < npairs; ++r, g += stride) {
            const uint64_t i = ((g & ~lowmask) << 1) | (g & lowmask);
            const uint64_t j = i ^ T.x;
            const Amp a = psi[i], b = psi[j];
            // w = a * conj(b)
            const R wr = a.x * b.x + a.y * b.y;
            const R wi = a.y * b.x - a.x * b.y;
            R e = 0;
            for (int k = 0; k < T.nt; ++k) {
                R v;
                switch (T.y4[k]) {
                case 0: v = wr; break;
                case 1: v = -wi; break;
                case 2: v = -wr; break;
                default: v = wi; break;
                }
                const R c = (R)T.c[k];
                e += (__popcll(i & T.z[k]) & 1) ? -c * v : c * v;
            }
            run += e;
        }
        acc += 2.0 * (double)run;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// ---------------------------------------------------------------------------
// full-register sampling
// ---------------------------------------------------------------------------
// Chunk sums: chunk b = [b*len, (b+1)*len), summed in FP64 over runs of 16
// terms per thread formed in the amplitude precision (16 loads in flight).
template <typename Amp>
__global__ void __launch_bounds__(kRedThreads) k_chunk_sums(const Amp *__restrict__ psi, uint64_t len,
                                                            double *__restrict__ sums) {
    typedef typename AmpTraits<Amp>::real R;
    __shared__ double sh[32];
    const Amp *p = psi + (uint64_t)blockIdx.x * len;
    double acc = 0.0;
    const uint64_t step = (uint64_t)blockDim.x * 16;
    for (uint64_t i0 = threadIdx.x; i0 < len; i0 += step) {
        R run = 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint64_t i = i0 + (uint64_t)u * blockDim.x;
            if (i < len) run += norm2(p[i]);
        }
        acc += (double)run;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

// Inclusive FP64 scan of |psi_i|^2 over one chunk, starting from `carry`;
// writes the first index whose running sum exceeds `target` (or ~0 if none)
// and that amplitude.  One block of 1024 threads; per step thread t owns the
// run of kSearchRun consecutive amplitudes at off + t * kSearchRun: run sums
// (FP64) are scanned across the block, and the one thread whose run crosses
// the target scans its own amplitudes.
struct SearchOut {
    unsigned long long index;
    double re, im;
    double total;
};

constexpr int kSearchThreads = 1024;
constexpr int kSearchRun = 32;

template <typename Amp>
__global__ void __launch_bounds__(kSearchThreads) k_chunk_search(const Amp *__restrict__ psi, uint64_t begin,
                                                                 uint64_t len, double carry, double target,
                                                                 SearchOut *out) {
    __shared__ double wsum[32];
    __shared__ unsigned long long found;
    __shared__ double s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        found = ~0ull;
        s_carry = carry;
    }
    __syncthreads();
    const uint64_t step = (uint64_t)kSearchThreads * kSearchRun;
    for (uint64_t off = 0; off < len; off += step) {
        const uint64_t r0 = off + (uint64_t)threadIdx.x * kSearchRun;  // this thread's run, relative to begin
        double run = 0.0;
        for (int k = 0; k < kSearchRun; ++k)
            if (r0 + k < len) run += (double)norm2(psi[begin + r0 + k]);
        // inclusive scan of the run sums over the block
        double w = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane == 31) wsum[warp] = w;
        __syncthreads();
        if (warp == 0) {
            double v = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            wsum[lane] = v;  // inclusive over warps
        }
        __syncthreads();
        const double before = s_carry + (warp > 0 ? wsum[warp - 1] : 0.0) + (w - run);  // sum ahead of this run
        if (r0 < len && before + run > target) {
            // the first crossing inside this run: the partial sums are formed
            // in the order of `run`, so the last one equals it and crosses
            double part = 0.0;
            uint64_t hit = r0;
            for (int k = 0; k < kSearchRun && r0 + k < len; ++k) {
                part += (double)norm2(psi[begin + r0 + k]);
                hit = r0 + k;
                if (before + part > target) break;
            }
            atomicMin(&found, (unsigned long long)(begin + hit));
        }
        __syncthreads();
        if (found != ~0ull) break;
        if (threadIdx.x == 0) s_carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->index = found;
        out->total = s_carry;
        if (found != ~0ull) {
            const Amp a = psi[found];
            out->re = (double)a.x;
            out->im = (double)a.y;
        }
    }
}

// Last index of non-zero weight in [begin, begin+len) (one block).
template <typename Amp>
__global__ void __launch_bounds__(1024) k_last_nonzero(const Amp *__restrict__ psi, uint64_t begin, uint64_t len,
                                                       SearchOut *out) {
    __shared__ unsigned long long best;
    if (threadIdx.x == 0) best = 0ull;
    __syncthreads();
    unsigned long long mine = 0ull;
    for (uint64_t off = threadIdx.x; off < len; off += blockDim.x)
        if (norm2(psi[begin + off]) > 0) mine = begin + off + 1;  // +1 so that 0 means none
    atomicMax(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        out->index = best ? best - 1 : ~0ull;
        if (best) {
            const Amp a = psi[best - 1];
            out->re = (double)a.x;
            out->im = (double)a.y;
        }
    }
}

template <typename Amp>
__global__ void k_write_basis(Amp *__restrict__ psi, uint64_t N, uint64_t j, double re, double im) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
        Amp z;
        z.x = (i == j) ? (typename AmpTraits<Amp>::real)re : 0;
        z.y = (i == j) ? (typename AmpTraits<Amp>::real)im : 0;
        psi[i] = z;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
InsertSpec make_spec(uint64_t mask) {
    InsertSpec s{};
    s.m = 0;
    for (int b = 0; b < 64; ++b)
        if ((mask >> b) & 1ull) s.pos[s.m++] = b;
    return s;
}

double *ws_partials(qsim *s) { return (double *)((char *)s->ws + kWsPartials); }
double *ws_result(qsim *s) { return (double *)((char *)s->ws + kWsResult); }
double *ws_chunks(qsim *s) { return (double *)((char *)s->ws + kWsChunk); }

unsigned grid_for(uint64_t work, int threads, unsigned cap) {
    const uint64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

// Copy `count` doubles from device to the pinned buffer and wait; also
// reports a raised device error flag.
int fetch(qsim *s, const double *dev, int count, double *host_out) {
    cudaError_t e = cudaMemcpyAsync(s->pinned, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "result copy");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "stream synchronize");
    std::memcpy(host_out, s->pinned, sizeof(double) * count);
    return check_device_errors(s);
}

int finalize(qsim *s, int nblocks, int V, double *host_out) {
    k_finalize<<<1, 64, 0, s->stream>>>(ws_partials(s), nblocks, V, ws_result(s));
    s->stats.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(s, e, "finalize launch");
    return fetch(s, ws_result(s), V, host_out);
}

template <typename Amp>
int probs_all_t(qsim *s, double *p1, double *norm2_out) {
    const int n = s->n;
    std::vector<double> v(n + 1);
    if (n < 10) {
        k_probs_small<Amp><<<1, 256, 0, s->stream>>>((const Amp *)s->state, n, ws_result(s));
        s->stats.launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(s, e, "probs launch");
        int rc = fetch(s, ws_result(s), n + 1, v.data());
        if (rc) return rc;
    } else {
        const uint64_t ntiles = 1ull << (n - 10);
        const unsigned grid = grid_for(ntiles, kRedThreads / 32, reduce_blocks(s));
        k_probs_tiles<Amp><<<grid, kRedThreads, 0, s->stream>>>((const Amp *)s->state, n, ntiles, ws_partials(s));
        s->stats.launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(s, e, "probs launch");
        int rc = finalize(s, grid, n + 1, v.data());
        if (rc) return rc;
    }
    if (norm2_out) *norm2_out = v[0];
    for (int q = 0; q < n; ++q) p1[q] = v[1 + q];
    return QSIM_OK;
}

// S0, S1 of qubit q by tiles (n >= 10); only_set: S1 alone, reading only
// the tiles with bit q set where q >= 10.
template <typename Amp>
int bit_sums_t(qsim *s, int q, bool only_set, double *s0, double *s1) {
    const int n = s->n;
    const uint64_t ntiles = (1ull << (n - 10)) >> ((only_set && q >= 10) ? 1 : 0);
    const unsigned grid = grid_for(ntiles, kRedThreads / 32, reduce_blocks(s));
    k_bit_sums<Amp><<<grid, kRedThreads, 0, s->stream>>>((const Amp *)s->state, q, ntiles, only_set ? 1 : 0,
                                                          ws_partials(s));
    s->stats.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(s, e, "bit sums launch");
    double v[2];
    int rc = finalize(s, grid, 2, v);
    if (rc) return rc;
    if (s0) *s0 = v[0];
    *s1 = v[1];
    return QSIM_OK;
}

template <typename Amp>
int masked_sum_t(qsim *s, uint64_t mask, uint64_t value, double *out) {
    if (s->n >= 10 && __builtin_popcountll(mask) == 1 && value == mask)
        return bit_sums_t<Amp>(s, __builtin_ctzll(mask), true, nullptr, out);
    const InsertSpec ins = make_spec(mask);
    const uint64_t ngroups = 1ull << (s->n - ins.m);
    const unsigned grid = grid_for(ngroups, kRedThreads, reduce_blocks(s));
    k_masked_sum<Amp><<<grid, kRedThreads, 0, s->stream>>>((const Amp *)s->state, ngroups, ins, value, ws_partials(s));
    s->stats.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(s, e, "masked sum launch");
    return finalize(s, grid, 1, out);
}

template <typename Amp>
int split_sum_t(qsim *s, int q, double *s0, double *s1) {
    if (s->n >= 10) return bit_sums_t<Amp>(s, q, false, s0, s1);
    const uint64_t npairs = 1ull << (s->n - 1);
    const unsigned grid = grid_for(npairs, kRedThreads, reduce_blocks(s));
    k_split_sum<Amp><<<grid, kRedThreads, 0, s->stream>>>((const Amp *)s->state, npairs, q, ws_partials(s));
    s->stats.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(s, e, "split sum launch");
    double v[2];
    int rc = finalize(s, grid, 2, v);
    if (rc) return rc;
    *s0 = v[0];
    *s1 = v[1];
    return QSIM_OK;
}

template <typename Amp>
int collapse_t(qsim *s, uint64_t mask, uint64_t value, double scale) {
    const uint64_t N = 1ull << s->n;
    const float shi = (float)scale;
    const float slo = (float)(scale - (double)shi);
    if (s->n >= 1 && __builtin_popcountll(mask) == 1) {
        const int q = __builtin_ctzll(mask);
        const uint64_t npairs = N >> 1;
        const unsigned grid = grid_for(npairs, 256, s->sms * 16);
        k_collapse_bit<Amp><<<grid, 256, 0, s->stream>>>((Amp *)s->state, npairs, q, value ? 1 : 0, scale, shi, slo);
        s->stats.launches++;
        return cuda_err(s, cudaGetLastError(), "collapse launch");
    }
    const unsigned grid = grid_for(N, 256, s->sms * 16);
    k_collapse_mask<Amp><<<grid, 256, 0, s->stream>>>((Amp *)s->state, N, mask, value, scale, shi, slo);
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "collapse launch");
}

template <typename Amp>
int expect_t(qsim *s, const qsim_pauli *terms, int nterms, double *out) {
    const int n = s->n;
    const uint64_t N = 1ull << n;
    double total = 0.0;
    // Z-only strings, in batches of kMaxZTerms
    std::vector<int> zonly;
    for (int k = 0; k < nterms; ++k)
        if (terms[k].xmask == 0) zonly.push_back(k);
    for (size_t b0 = 0; b0 < zonly.size(); b0 += kMaxZTerms) {
        ZTerms T{};
        T.nt = (int)std::min<size_t>(kMaxZTerms, zonly.size() - b0);
        // group the batch's terms by their bits inside a tile (0..9)
        std::vector<int> ord(T.nt);
        for (int k = 0; k < T.nt; ++k) ord[k] = zonly[b0 + k];
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return (terms[a].zmask & 0x3FFull) < (terms[b].zmask & 0x3FFull); });
        T.ng = 0;
        for (int k = 0; k < T.nt; ++k) {
            const uint64_t z = terms[ord[k]].zmask;
            if (k == 0 || (z & 0x3FFull) != (terms[ord[k - 1]].zmask & 0x3FFull)) {
                T.first[T.ng] = k;
                T.zl[T.ng] = (int)(z & 31u);
                T.m[T.ng] = (int)((z >> 5) & 31u);
                ++T.ng;
            }
            T.c[k] = terms[ord[k]].coeff;
            T.cf[k] = (float)terms[ord[k]].coeff;
            T.zh[k] = (unsigned)(z >> 10);
        }
        T.first[T.ng] = T.nt;
        double v;
        if (n < 10) {
            k_expect_z_small<Amp><<<1, 256, 0, s->stream>>>((const Amp *)s->state, N, T, ws_result(s));
            s->stats.launches++;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_err(s, e, "expect launch");
            int rc = fetch(s, ws_result(s), 1, &v);
            if (rc) return rc;
        } else {
            const uint64_t ntiles = 1ull << (n - 10);
            const unsigned grid = grid_for(ntiles, kZThreads / 32, 2 * reduce_blocks(s));
            k_expect_z_tiles<Amp><<<grid, kZThreads, 0, s->stream>>>((const Amp *)s->state, ntiles, T,
                                                                         ws_partials(s));
            s->stats.launches++;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_err(s, e, "expect launch");
            int rc = finalize(s, grid, 1, &v);
            if (rc) return rc;
        }
        total += v;
    }
    // strings with an X part, grouped by X mask
    std::vector<int> rest;
    for (int k = 0; k < nterms; ++k)
        if (terms[k].xmask != 0) rest.push_back(k);
    std::stable_sort(rest.begin(), rest.end(), [&](int a, int b) { return terms[a].xmask < terms[b].xmask; });
    size_t i = 0;
    while (i < rest.size()) {
        XTerms T{};
        T.x = terms[rest[i]].xmask;
        T.h = 63 - __builtin_clzll(T.x);
        T.nt = 0;
        while (i < rest.size() && terms[rest[i]].xmask == T.x && T.nt < kMaxXTerms) {
            const qsim_pauli &p = terms[rest[i]];
            T.c[T.nt] = p.coeff;
            T.z[T.nt] = p.zmask;
            T.y4[T.nt] = __builtin_popcountll(p.xmask & p.zmask) & 3;
            ++T.nt;
            ++i;
        }
        const uint64_t npairs = N >> 1;
        const unsigned grid = grid_for(npairs, kRedThreads, reduce_blocks(s));
        k_expect_x<Amp><<<grid, kRedThreads, 0, s->stream>>>((const Amp *)s->state, npairs, T, ws_partials(s));
        s->stats.launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(s, e, "expect launch");
        double v;
        int rc = finalize(s, grid, 1, &v);
        if (rc) return rc;
        total += v;
    }
    *out = total;
    return QSIM_OK;
}

template <typename Amp>
int measure_all_t(qsim *s, double u, uint64_t *outcome) {
    const int n = s->n;
    const uint64_t N = 1ull << n;
    const int nchunks = (int)std::min<uint64_t>(kMaxChunks, std::max<uint64_t>(1, N >> 8));
    const uint64_t len = N / (uint64_t)nchunks;
    k_chunk_sums<Amp><<<nchunks, kRedThreads, 0, s->stream>>>((const Amp *)s->state, len, ws_chunks(s));
    s->stats.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(s, e, "chunk sums launch");
    e = cudaMemcpyAsync(s->pinned, ws_chunks(s), sizeof(double) * nchunks, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "chunk sums copy");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "stream synchronize");
    std::vector<double> sums(s->pinned, s->pinned + nchunks);
    double norm = 0.0;
    for (double v : sums) norm += v;
    if (!(norm > 0.0)) return set_err(s, QSIM_EZEROPROB, "measure_all on a zero vector");
    const double target = u * norm;
    SearchOut *dout = (SearchOut *)ws_result(s);
    SearchOut res{};
    double prefix = 0.0;
    int b = 0;
    bool done = false;
    for (; b < nchunks && !done; ++b) {
        if (sums[b] > 0.0 && prefix + sums[b] > target) {
            k_chunk_search<Amp><<<1, kSearchThreads, 0, s->stream>>>((const Amp *)s->state, (uint64_t)b * len, len, prefix,
                                                           target, dout);
            s->stats.launches++;
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_err(s, e, "chunk search launch");
            double tmp[4];
            int rc = fetch(s, (const double *)dout, 4, tmp);
            if (rc) return rc;
            std::memcpy(&res, tmp, sizeof(res));
            if (res.index != ~0ull) done = true;
        }
        prefix += sums[b];
    }
    if (!done) {
        // rounding left no index above the target: take the last one of
        // non-zero weight
        int last = nchunks - 1;
        while (last > 0 && !(sums[last] > 0.0)) --last;
        k_last_nonzero<Amp><<<1, 1024, 0, s->stream>>>((const Amp *)s->state, (uint64_t)last * len, len, dout);
        s->stats.launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(s, e, "last nonzero launch");
        double tmp[4];
        int rc = fetch(s, (const double *)dout, 4, tmp);
        if (rc) return rc;
        std::memcpy(&res, tmp, sizeof(res));
        if (res.index == ~0ull) return set_err(s, QSIM_EZEROPROB, "no amplitude of non-zero weight");
    }
    const double mag = std::sqrt(res.re * res.re + res.im * res.im);
    const unsigned grid = grid_for(N, 256, s->sms * 16);
    k_write_basis<Amp><<<grid, 256, 0, s->stream>>>((Amp *)s->state, N, res.index, res.re / mag, res.im / mag);
    s->stats.launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(s, e, "collapse to basis launch");
    *outcome = res.index;
    return QSIM_OK;
}

}  // namespace

int run_probs_all(qsim *s, double *p1, double *norm2) {
    return s->prec == QSIM_C128 ? probs_all_t<double2>(s, p1, norm2) : probs_all_t<float2>(s, p1, norm2);
}
int run_masked_sum(qsim *s, uint64_t mask, uint64_t value, double *out) {
    return s->prec == QSIM_C128 ? masked_sum_t<double2>(s, mask, value, out)
                                : masked_sum_t<float2>(s, mask, value, out);
}
int run_split_sum(qsim *s, int q, double *s0, double *s1) {
    return s->prec == QSIM_C128 ? split_sum_t<double2>(s, q, s0, s1) : split_sum_t<float2>(s, q, s0, s1);
}
int run_collapse_mask(qsim *s, uint64_t mask, uint64_t value, double scale) {
    return s->prec == QSIM_C128 ? collapse_t<double2>(s, mask, value, scale) : collapse_t<float2>(s, mask, value, scale);
}
int run_expect(qsim *s, const qsim_pauli *terms, int nterms, double *out) {
    return s->prec == QSIM_C128 ? expect_t<double2>(s, terms, nterms, out) : expect_t<float2>(s, terms, nterms, out);
}
int run_measure_all(qsim *s, double u, uint64_t *outcome) {
    return s->prec == QSIM_C128 ? measure_all_t<double2>(s, u, outcome) : measure_all_t<float2>(s, u, outcome);
}

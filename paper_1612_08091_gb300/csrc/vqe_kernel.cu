// vqe_kernel.cu -- a batch of variational circuits in one persistent launch.
//
// Not a method of the paper: the serving pattern of many small
// hardware-efficient-ansatz circuits (different qubit counts and depths)
// evaluated together, each ending in the transverse-field Ising energy
//   E = -sum_{i<n-1} <Z_i Z_{i+1}> - h sum_i <X_i>   (open chain).
// A circuit starts in |0...0> and runs L layers of RY(theta_q) on every
// qubit, RZ(phi_q) on every qubit, then CNOT(q -> q+1) for q = 0..n-2.
//
// Per layer the two rotations on a qubit fuse into U_q = RZ(phi) RY(theta)
// (they commute with the rotations on the other qubits), and the CNOT
// ladder is one permutation: applied in order it maps |b> to |b'> with
// b'_k = b_0 ^ ... ^ b_k, i.e. psi'[y] = psi[y ^ (y << 1) mod 2^n].
//
// One persistent launch: every CTA takes circuit ids from an atomic counter
// (largest circuits first) until the batch is done; there is no waiting on
// other CTAs.  A circuit of n <= m qubits (m = 12..14, tuned) lives in the
// CTA's shared memory; a larger one lives in a per-CTA pair of global
// buffers and is processed in chunks of 2^g amplitudes (g = 12):
//   pair pass: the ladder permutation of the previous layer maps the
//     destination chunks hi and hi ^ (2^h - 1) (h = n - g) onto the same two
//     source chunks S, S ^ 1 with S = hi ^ (hi << 1): an element at offset o
//     of source chunk S ^ p lands in chunk hi if parity(o) == p, else in its
//     partner, at the offset whose bit k is the XOR of bits 0..k of o.  Both
//     source chunks are copied whole into shared memory and stay in source
//     order there (logical qubit k pairs the elements p and p ^ (3 << k)),
//     get the gates on qubits 0..g-1, and are written back whole, each
//     destination element read from its source position;
//   high pass: tiles made of runs of 2^(g-h) amplitudes times the h top
//     qubits get the gates on the top qubits, in place.
// The energy is read after one more pair pass that applies the last layer's
// permutation.  Amplitudes are complex64 in FP32 arithmetic; energies
// accumulate per thread in FP32 over a few terms and in FP64 beyond.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/qsim.h"
#include "common.cuh"
#include "tc_common.cuh"

using namespace qsim_dev;
using namespace qsim_tc;

namespace {

// amplitudes per thread held in registers for the in-place permutation
template <int T> struct RegAmps { static constexpr int value = T >= 1024 ? 16 : 32; };

struct VqeArgs {
    const int *order;
    const int *nq;
    const int *nl;
    const long long *aoff;
    const double *angles;
    double *energies;
    unsigned int *counter;  // this launch's queue
    unsigned int *err;      // error flag (a bounded wait gave up)
    int begin, end;   // its circuits: order[begin..end)
    int m;            // qubits held in shared memory
    float2 *gbuf;     // per-CTA global buffers (two of gstride amplitudes each)
    size_t gstride;
    double h;
};

// A layer's rotations factor as (prod_q RZ(phi_q)) (prod_q RY(theta_q)):
// RZ and RY on one qubit keep their order, and gates on different qubits
// commute.  Write theta/2 = theta'/2 + j pi/2 with |theta'/2| <= pi/4; then
//   RY(theta) = RY(j pi) RY(theta'),   RY(pi) = X Z,   RY(2 pi) = -I,
//   RY(theta') = c' [[1, -t], [t, 1]],  c' = cos(theta'/2), t = tan(theta'/2),
// so the rotation proper is two FMAs per amplitude (|t| <= 1) and the rest
// is bookkeeping: c' and the sign (-1)^floor(j/2) join the layer's global
// factor, and for odd j the X Z is moved past the RZ (RZ(phi) X = X RZ(-phi)):
//   RZ(phi) RY(theta) = s c' X diag(e^{i phi/2}, -e^{-i phi/2}) [[1, -t], [t, 1]].
// The diagonal part of all qubits is
//   exp(-i Phi'/2) prod_{q in i} p_q,  p_q = e^{i phi_q} or -e^{-i phi_q} (odd j),
// Phi' = sum_q (+-phi_q), applied as one complex factor per amplitude from
// two small tables (low and high bits) while the amplitudes move anyway, and
// the X of the qubits with odd j (the layer's flip mask F) is an XOR of the
// index where each amplitude is read for writing back.
struct Rot {
    float t;
};

__device__ __forceinline__ void apply_pair(float2 *x, unsigned i0, unsigned i1, const Rot &g) {
    const float2 a = x[i0], b = x[i1];
    x[i0] = make_float2(fmaf(-g.t, b.x, a.x), fmaf(-g.t, b.y, a.y));
    x[i1] = make_float2(fmaf(g.t, a.x, b.x), fmaf(g.t, a.y, b.y));
}

// Rotation pairing the elements i and i ^ mask of a 2^k-amplitude array in
// shared memory (mask's lowest bit, the pivot, is 0 in i).
__device__ __forceinline__ void gate_smem(float2 *x, int k, unsigned mask, const Rot &g) {
    const unsigned half = 1u << (k - 1);
    const unsigned lowmask = (mask & (0u - mask)) - 1u;
    for (unsigned p = threadIdx.x; p < half; p += blockDim.x) {
        const unsigned i0 = ((p & ~lowmask) << 1) | (p & lowmask);
        apply_pair(x, i0, i0 ^ mask, g);
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned ladder_src(unsigned y, unsigned mask) { return (y ^ (y << 1)) & mask; }

// Rotations g[0..nb) on a 2^k-amplitude array in shared memory, applied four
// at a time in registers: each thread loads the 16 amplitudes of a group,
// applies the four rotations there and stores them back, so a layer of k
// one-qubit rotations costs ceil(k/4) passes over shared memory instead of k.
// Rotation j pairs the elements i and i ^ mask[j] (single bits here; the
// pair pass of the global-memory path, whose buffers are in source order,
// has its own compile-time version, pair_group).  The masks' bits must
// differ; a group is a base with zeros at its bits XOR any subset of its
// masks.  A group of fewer than four rotations is padded with identity
// rotations on other bits.
__device__ __forceinline__ void cswap(int &a, int &b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

__device__ void gates_blocked(float2 *x, int k, const unsigned *mask, const Rot *g, int nb) {
    if (k < 4) {
        // fewer than four bits in the array: one pass per gate
        for (int j = 0; j < nb; ++j) gate_smem(x, k, mask[j], g[j]);
        return;
    }
    for (int g0 = 0; g0 < nb; g0 += 4) {
        // the group's four bits (padded with identity gates on the lowest
        // unused bits)
        const bool h1 = g0 + 1 < nb, h2 = g0 + 2 < nb, h3 = g0 + 3 < nb;
        unsigned m0 = mask[g0], m1 = h1 ? mask[g0 + 1] : 0u, m2 = h2 ? mask[g0 + 2] : 0u,
                 m3 = h3 ? mask[g0 + 3] : 0u;
        unsigned used = (m0 & (0u - m0)) | (m1 & (0u - m1)) | (m2 & (0u - m2)) | (m3 & (0u - m3));
        // padding on the lowest unused bit, at bit 4 or above where one is
        // free (a pivot in bits 0..3, the bank bits, costs a bank conflict)
        auto pad = [&]() {
            const unsigned hi = ~used & ((1u << k) - 1u) & ~15u;
            const unsigned m = hi ? (hi & (0u - hi)) : (~used & (used + 1u));
            used |= m;
            return m;
        };
        if (!h1) m1 = pad();
        if (!h2) m2 = pad();
        if (!h3) m3 = pad();
        const float t0 = g[g0].t, t1 = h1 ? g[g0 + 1].t : 0.f, t2 = h2 ? g[g0 + 2].t : 0.f,
                    t3 = h3 ? g[g0 + 3].t : 0.f;
        int s0 = __ffs(m0) - 1, s1 = __ffs(m1) - 1, s2 = __ffs(m2) - 1, s3 = __ffs(m3) - 1;
        cswap(s0, s1);
        cswap(s2, s3);
        cswap(s0, s2);
        cswap(s1, s3);
        cswap(s1, s2);
        const unsigned ngroups = 1u << (k - 4);
        for (unsigned gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
            unsigned base = gi;
            base = ((base >> s0) << (s0 + 1)) | (base & ((1u << s0) - 1u));
            base = ((base >> s1) << (s1 + 1)) | (base & ((1u << s1) - 1u));
            base = ((base >> s2) << (s2 + 1)) | (base & ((1u << s2) - 1u));
            base = ((base >> s3) << (s3 + 1)) | (base & ((1u << s3) - 1u));
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r)
                v[r] = x[base ^ ((r & 1) ? m0 : 0u) ^ ((r & 2) ? m1 : 0u) ^ ((r & 4) ? m2 : 0u) ^ ((r & 8) ? m3 : 0u)];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float t = j == 0 ? t0 : j == 1 ? t1 : j == 2 ? t2 : t3;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    if ((r >> j) & 1) continue;
                    const int r1 = r | (1 << j);
                    const float2 a = v[r], bb = v[r1];
                    v[r] = make_float2(fmaf(-t, bb.x, a.x), fmaf(-t, bb.y, a.y));
                    v[r1] = make_float2(fmaf(t, a.x, bb.x), fmaf(t, a.y, bb.y));
                }
            }
#pragma unroll
            for (int r = 0; r < 16; ++r)
                x[base ^ ((r & 1) ? m0 : 0u) ^ ((r & 2) ? m1 : 0u) ^ ((r & 4) ? m2 : 0u) ^ ((r & 8) ? m3 : 0u)] = v[r];
        }
        __syncthreads();
    }
}

__device__ double block_sum_d(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
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

// ZZ part of a 2^k chunk whose global index bits above k are `hi` (n qubits):
// sum_i |psi_i|^2 * ((n-1) - 2 popc((i ^ i>>1) & (2^(n-1)-1))).
__device__ float zz_chunk(const float2 *x, int k, unsigned long long hi, int n) {
    const unsigned long long m1 = (n >= 2) ? ((1ull << (n - 1)) - 1ull) : 0ull;
    float acc = 0.f;
    for (unsigned i = threadIdx.x; i < (1u << k); i += blockDim.x) {
        const unsigned long long gi = hi | i;
        const float w = norm2(x[i]);
        acc += w * (float)((n - 1) - 2 * __popcll((gi ^ (gi >> 1)) & m1));
    }
    return acc;
}

// sum over pairs on bit `bit` of 2 Re(conj(a) b) inside a 2^k array
__device__ float x_chunk(const float2 *x, int k, int bit) {
    const unsigned half = 1u << (k - 1);
    const unsigned lowmask = (1u << bit) - 1u;
    float acc = 0.f;
    for (unsigned p = threadIdx.x; p < half; p += blockDim.x) {
        const unsigned i0 = ((p & ~lowmask) << 1) | (p & lowmask);
        const float2 a = x[i0], b = x[i0 | (1u << bit)];
        acc += 2.f * (a.x * b.x + a.y * b.y);
    }
    return acc;
}

// t[j] = extra * prod over the set bits i of j (i < kb) of ph[i]
__device__ void build_phase_table(float2 *t, int kb, const float2 *ph, float2 extra) {
    for (unsigned j = threadIdx.x; j < (1u << kb); j += blockDim.x) {
        float2 z = extra;
        for (int i = 0; i < kb; ++i)
            if ((j >> i) & 1u) z = cmul(z, ph[i]);
        t[j] = z;
    }
}

// GLOBAL = false: circuits of n <= m qubits, each held in one CTA's shared
// memory.  GLOBAL = true: larger circuits in per-CTA global buffers, two
// CTAs per SM so that one CTA's loads, arithmetic and stores overlap the
// other's (measured faster than one CTA of 512 threads per SM with
// double-buffered copies: 44.9 against 41.0 ms for the 4096-circuit batch).
// The global-memory kernel's chunk size (2^12 amplitudes; a pair of chunks
// is 64 KB of shared memory) and block size.
constexpr int kGlobalThreads = 128;
constexpr int kGlobalCtas = 3;  // resident CTAs per SM the register budget is sized for
constexpr int kGlobalBits = 12;

// Position in a pair buffer (source order, after a ladder permutation) of
// logical element e: bits 0..g-1 are gl = (e ^ e << 1) mod 2^g, bit g is
// parity(gl) ^ (e >> g).  The map is linear over GF(2), so for the store's
// elements e = tid ^ (j << 8) it is pair_perm(tid) ^ pair_perm(j << 8), the
// second term a compile-time constant.
__host__ __device__ constexpr unsigned pair_perm(unsigned e) {
    const unsigned gl = (e ^ (e << 1)) & ((1u << kGlobalBits) - 1u);
    unsigned par = 0;
    for (int b = 0; b < kGlobalBits; ++b) par ^= (gl >> b) & 1u;
    return ((par ^ (e >> kGlobalBits)) << kGlobalBits) | gl;
}

// Order of the pair pass's 12 rotations, taken four at a time, one of the
// qubits 0..2 in each group (qubits 0..3 decide the shared-memory bank of
// an 8-byte element; see pair_group for how the groups avoid conflicts).
__constant__ int kPairOrder[12] = {0, 4, 5, 6, 1, 7, 8, 9, 2, 3, 10, 11};

// One group of the pair pass with compile-time qubits Q0 < Q1 < Q2 < Q3 (a
// group of kPairOrder): the 2^13-element pair buffer x holds 512 groups of
// 16 elements, base (zeros at the pivots P0 < P1 < P2 < P3) XOR any subset
// of the masks Mj = (PERM ? 3 : 1) << Qj; rotation j uses r[j].t.  PERM: the
// buffer is in source order after a ladder permutation, where logical qubit
// k pairs the elements p and p ^ (3 << k); either of those two bits can be
// the pivot (Pj = Qj or Qj + 1; the masks restricted to the pivots must be
// invertible); the element whose logical bit k is 0 is the one whose bits
// 0..k have even parity, which for rotation j is the base's parity, so the
// rotation is applied with t -> -t where that parity is odd.
//
// Banks.  In each access all lanes use the same subset of masks, so the 16
// lanes of a half-warp (8-byte elements) hit 16 banks only if their bases
// differ in all of bits 0..3.  A pivot there is 0 in every base; instead,
// lanes whose group-index bit (4 - c + i) is set (c = number of pivots
// below 4) start from base ^ M of the i-th such rotation: the same 16
// elements in another order, which flips that pivot's bank bit, and that
// rotation's pair is met with its two elements swapped (t -> -t in those
// lanes).  The other rotations are unaffected: a mask changes the parity of
// bits 0..q of no other rotation's base.
template <bool PERM, int Q0, int Q1, int Q2, int Q3, int P0, int P1, int P2, int P3>
__device__ __forceinline__ void pair_group(float2 *x, const Rot *r) {
    static_assert(Q0 < Q1 && Q1 < Q2 && Q2 < Q3, "qubits in ascending order");
    static_assert(P0 < P1 && P1 < P2 && P2 < P3, "pivots in ascending order");
    constexpr unsigned W = PERM ? 3u : 1u;
    constexpr unsigned M0 = W << Q0, M1 = W << Q1, M2 = W << Q2, M3 = W << Q3;
    static_assert(((M0 >> P0) & 1u) && ((M1 >> P1) & 1u) && ((M2 >> P2) & 1u) && ((M3 >> P3) & 1u),
                  "each pivot is a bit of its own mask");
    // restricted to the pivots the masks form a triangular matrix
    static_assert(!((M0 >> P1) & 1u) && !((M0 >> P2) & 1u) && !((M0 >> P3) & 1u) && !((M1 >> P2) & 1u) &&
                      !((M1 >> P3) & 1u) && !((M2 >> P3) & 1u) ||
                  (!((M1 >> P0) & 1u) && !((M2 >> P0) & 1u) && !((M3 >> P0) & 1u) && !((M2 >> P1) & 1u) &&
                   !((M3 >> P1) & 1u) && !((M3 >> P2) & 1u)),
                  "masks restricted to the pivots must be invertible");
    constexpr int c = (P0 < 4) + (P1 < 4) + (P2 < 4) + (P3 < 4);  // pivots in the bank bits
    static_assert(c <= 2 && (P0 < 4 || c == 0) && (P1 < 4 || c <= 1) && P2 >= 4 && P3 >= 4,
                  "bank pivots come first");
    const float t0 = r[0].t, t1 = r[1].t, t2 = r[2].t, t3 = r[3].t;
    for (unsigned gi = threadIdx.x; gi < (1u << (kGlobalBits + 1 - 4)); gi += (unsigned)kGlobalThreads) {
        unsigned base = gi;
        base = ((base >> P0) << (P0 + 1)) | (base & ((1u << P0) - 1u));
        base = ((base >> P1) << (P1 + 1)) | (base & ((1u << P1) - 1u));
        base = ((base >> P2) << (P2 + 1)) | (base & ((1u << P2) - 1u));
        base = ((base >> P3) << (P3 + 1)) | (base & ((1u << P3) - 1u));
        // lane-dependent start of the bank-pivot rotations (see above)
        const bool sw0 = c >= 1 && ((gi >> (4 - c)) & 1u);
        const bool sw1 = c >= 2 && ((gi >> (5 - c)) & 1u);
        const unsigned start = base ^ (sw0 ? M0 : 0u) ^ (sw1 ? M1 : 0u);
        float2 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
            v[k] = x[start ^ ((k & 1) ? M0 : 0u) ^ ((k & 2) ? M1 : 0u) ^ ((k & 4) ? M2 : 0u) ^ ((k & 8) ? M3 : 0u)];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = j == 0 ? Q0 : j == 1 ? Q1 : j == 2 ? Q2 : Q3;
            float t = j == 0 ? t0 : j == 1 ? t1 : j == 2 ? t2 : t3;
            if (PERM && (__popc(base & ((2u << q) - 1u)) & 1)) t = -t;
            if ((j == 0 && sw0) || (j == 1 && sw1)) t = -t;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if ((k >> j) & 1) continue;
                const int k1 = k | (1 << j);
                const float2 a = v[k], b = v[k1];
                v[k] = make_float2(fmaf(-t, b.x, a.x), fmaf(-t, b.y, a.y));
                v[k1] = make_float2(fmaf(t, a.x, b.x), fmaf(t, a.y, b.y));
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            x[start ^ ((k & 1) ? M0 : 0u) ^ ((k & 2) ? M1 : 0u) ^ ((k & 4) ? M2 : 0u) ^ ((k & 8) ? M3 : 0u)] = v[k];
    }
    __syncthreads();
}

// The pair pass's 12 rotations (r in kPairOrder) on a pair buffer.  Group
// {2, 3, 10, 11} takes qubit 3's pivot at bit 4 when PERM allows it, so that
// it has one pivot in the bank bits, like the other two groups.
template <bool PERM>
__device__ __forceinline__ void pair_gates(float2 *x, const Rot *r) {
    pair_group<PERM, 0, 4, 5, 6, 0, 4, 5, 6>(x, r);
    pair_group<PERM, 1, 7, 8, 9, 1, 7, 8, 9>(x, r + 4);
    pair_group<PERM, 2, 3, 10, 11, 2, (PERM ? 4 : 3), 10, 11>(x, r + 8);
}

template <int T, bool GLOBAL>
__global__ void __launch_bounds__(T, GLOBAL ? kGlobalCtas : 1) k_vqe_batch(const VqeArgs A) {
    constexpr int kRegAmps = RegAmps<T>::value;
    extern __shared__ float2 sm[];
    __shared__ int s_idx;
    __shared__ double s_red[32];
    __shared__ Rot s_rot[32];       // this layer's RY per qubit
    __shared__ Rot s_rotp[32];      // the pair pass's rotations, in kPairOrder
    __shared__ float2 s_ph[32];     // e^{i phi_q}
    __shared__ unsigned s_mask[32]; // XOR mask of each rotation in the current pass
    __shared__ float2 s_tlo[128];   // phases of index bits 0..6 (times the global factor)
    __shared__ float2 s_thi[128];   // phases of the next bits of a chunk or register
    __shared__ float2 s_gph;        // the layer's global factor: prod_q s_q c'_q times e^{-i Phi'/2}
    __shared__ unsigned s_flip;     // the layer's flip mask F
    __shared__ __align__(8) uint64_t s_bar[1];  // bulk-copy completion (global-memory path)
    __shared__ uint32_t s_phase;
    if (threadIdx.x == 0) {
        if (GLOBAL) {
            mbar_init(s_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            s_phase = 0;
        }
    }
    __syncthreads();
    // the layer's rotations t_q, per-qubit phases p_q, flip mask and global
    // factor (warp 0; n <= 32)
    auto layer_setup = [&](const double *al, int n) {
        if (threadIdx.x < 32) {
            const unsigned q = threadIdx.x;
            unsigned flip = 0;
            float2 f = make_float2(1.f, 0.f);
            if (q < (unsigned)n) {
                constexpr double kPi = 3.14159265358979323846;
                const double hth = remainder(0.5 * al[q], 2.0 * kPi);  // theta/2 (RY has period 4 pi)
                const double j = rint(hth * (2.0 / kPi));                // -2..2
                const int ji = (int)j;
                float sh, ch;
                sincosf((float)(hth - j * (0.5 * kPi)), &sh, &ch);
                flip = (unsigned)ji & 1u;
                const float sc = ((ji >> 1) & 1) ? -ch : ch;  // (-1)^floor(j/2) c'
                const double phi = al[n + q];
                float sp, cp, s2, c2;
                sincosf((float)remainder(phi, 2.0 * kPi), &sp, &cp);
                sincosf((float)(0.5 * remainder(phi, 4.0 * kPi)), &s2, &c2);
                s_rot[q] = Rot{sh / ch};
                s_ph[q] = flip ? make_float2(-cp, sp) : make_float2(cp, sp);
                f = make_float2(sc * c2, flip ? sc * s2 : -sc * s2);
            }
            const unsigned fl = __ballot_sync(0xffffffffu, flip);
#pragma unroll
            for (int o = 16; o; o >>= 1)
                f = cmul(f, make_float2(__shfl_xor_sync(0xffffffffu, f.x, o), __shfl_xor_sync(0xffffffffu, f.y, o)));
            if (q == 0) {
                s_gph = f;
                s_flip = fl;
            }
        }
        __syncthreads();
    };
    for (;;) {
        if (threadIdx.x == 0) s_idx = A.begin + (int)atomicAdd(A.counter, 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= A.end) break;
        const int c = A.order[idx];
        const int n = A.nq[c], L = A.nl[c];
        const double *ang = A.angles + A.aoff[c];
        const unsigned N = 1u << n;
        double zz = 0.0, xx = 0.0;
        if constexpr (!GLOBAL) {
            // --- shared-memory resident circuit -------------------------------
            for (unsigned i = threadIdx.x; i < N; i += T) sm[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
            __syncthreads();
            const int klo = n < 7 ? n : 7;
            for (int l = 0; l < L; ++l) {
                const double *al = ang + 2 * l * n;
                if (threadIdx.x < (unsigned)n) s_mask[threadIdx.x] = 1u << threadIdx.x;
                layer_setup(al, n);
                build_phase_table(s_tlo, klo, s_ph, s_gph);
                build_phase_table(s_thi, n - klo, s_ph + klo, make_float2(1.f, 0.f));
                gates_blocked(sm, n, s_mask, s_rot, n);  // ends with a barrier
                // the RZ phases, the flips and the CNOT ladder as one pass
                // through registers
                const unsigned F = s_flip;
                float2 v[kRegAmps];
#pragma unroll
                for (int j = 0; j < kRegAmps; ++j) {
                    const unsigned y = threadIdx.x + (unsigned)j * T;
                    if (y < N) {
                        const unsigned x = ladder_src(y, N - 1) ^ F;
                        v[j] = cmul(sm[x], cmul(s_tlo[x & 127u], s_thi[x >> 7]));
                    }
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < kRegAmps; ++j) {
                    const unsigned y = threadIdx.x + (unsigned)j * T;
                    if (y < N) sm[y] = v[j];
                }
                __syncthreads();
            }
            zz = (double)zz_chunk(sm, n, 0ull, n);
            for (int q = 0; q < n; ++q) xx += (double)x_chunk(sm, n, q);
        } else {
            // --- global-memory circuit, chunks of 2^g ----------------------------
            // Data arrive by bulk copies completing on an mbarrier (no
            // register staging): a pair pass copies the two source chunks
            // whole and works on them in source order, where logical qubit
            // k < g pairs the elements p and p ^ (3 << k); the store reads
            // each destination element at its source position.  Every wait
            // is bounded; on time-out the CTA raises the error flag and
            // stops.
            constexpr int g = kGlobalBits;
            // the top-qubit pass takes tiles of the whole pair buffer, 2^(g+1)
            // amplitudes: 2^h runs of 2^lowrun (h >= 1, lowrun >= 1 for n <= 2g)
            const int h = n - g, lowrun = g + 1 - h;
            float2 *src = A.gbuf + (size_t)blockIdx.x * 2 * A.gstride;
            float2 *dst = src + A.gstride;
            const unsigned G = 1u << g, nchunks = 1u << h, hmask = nchunks - 1u, gmask = G - 1u;
            const unsigned run_bytes = 8u << lowrun;  // a high-pass tile is 2^h runs of 2^lowrun amplitudes
            const unsigned ntiles = nchunks / 2, GT = 2u * G;
            float2 *const s_ttop = sm + ((size_t)2 << g);  // phases of the top h qubits, after the pair buffer
            for (unsigned i = threadIdx.x; i < N; i += T) src[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
            __syncthreads();
            bool permuted = false;  // src holds the state before a pending ladder permutation
            bool failed = false;
            // wait for the current copy phase; the result is uniform over the CTA
            auto wait_copies = [&]() {
                bool ok = mbar_wait(s_bar, s_phase);
                if (!ok) ok = mbar_wait(s_bar, s_phase);  // give copies in flight a second bound
                __syncthreads();
                if (threadIdx.x == 0) s_phase ^= 1u;
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) atomicOr(A.err, 1u);
                    return false;
                }
                return true;
            };
            // chunks pr and pr ^ hmask (through the pending permutation: the
            // source chunks S and S ^ 1, S = pr ^ (pr << 1)) into sm[0..2G)
            // every thread orders its generic stores to global memory and its
            // shared-memory accesses before the bulk copies that follow
            auto before_copies = [&]() {
                fence_proxy_async_global();
                fence_proxy_async_smem();
                __syncthreads();
            };
            // the two source chunks of destination pair pr
            auto pair_chunks = [&](unsigned pr, unsigned &ca, unsigned &cb) {
                const unsigned S = permuted ? ((pr ^ (pr << 1)) & hmask) : pr;
                ca = S;
                cb = permuted ? S ^ 1u : pr ^ hmask;
            };
            // (Bringing the next pair's or tile's data into L2 once a copy
            // had landed, with cp.async.bulk.prefetch.L2, measured 4 %
            // slower: 6.5 % more DRAM reads.)
            auto load_pair = [&](const float2 *from, unsigned pr) {
                unsigned ca, cb;
                pair_chunks(pr, ca, cb);
                before_copies();
                if (threadIdx.x == 0) {
                    mbar_expect_tx(s_bar, 16u * G);
                    bulk_copy(sm, from + ((size_t)ca << g), 8u * G, s_bar);
                    bulk_copy(sm + G, from + ((size_t)cb << g), 8u * G, s_bar);
                }
                return wait_copies();
            };
            // physical position in the pair buffer of logical element e
            // (e < G: chunk pr, else chunk pr ^ hmask; offset e & gmask)
            auto pair_pos = [&](unsigned e) {
                if (!permuted) return e;
                const unsigned gl = ((e ^ (e << 1)) & gmask);
                return ((((unsigned)__popc(gl) & 1u) ^ (e >> g)) << g) | gl;
            };
            // Destination chunks pr (logical elements e < G) and pr ^ hmask,
            // written whole: this thread's elements are e = tid + j T, each
            // read at pair_pos(e ^ flo) (linear: a per-thread part and a
            // compile-time part); phased: the layer's phases of qubits
            // 0..g-1 and flips (flo), the low seven phase bits constant per
            // thread.
            auto store_pair = [&](float2 *to, unsigned pr, bool phased, unsigned flo) {
                static_assert(T == kGlobalThreads && T >= 128 && (2 << g) % T == 0,
                              "store_pair: the thread index holds bits 0..6 of the element");
                const unsigned tf = threadIdx.x ^ flo;
                const unsigned pt = permuted ? pair_perm(tf) : tf;
                float2 *dst0 = to + ((size_t)pr << g) + threadIdx.x;
                float2 *dst1 = to + ((size_t)(pr ^ hmask) << g) + threadIdx.x;
                const float2 tlo = s_tlo[tf & 127u];
                const unsigned thi0 = (tf >> 7) & 31u;
#pragma unroll
                for (int j = 0; j < (2 << g) / T; ++j) {
                    const unsigned cj = (unsigned)j * (unsigned)T;  // e = tid | j T
                    float2 v = sm[pt ^ (permuted ? pair_perm(cj) : cj)];
                    if (phased) v = cmul(v, cmul(tlo, s_thi[thi0 ^ ((cj >> 7) & 31u)]));
                    ((j < G / T) ? dst0 : dst1)[cj & gmask] = v;
                }
                __syncthreads();
            };
            auto tile_index = [&](unsigned t, unsigned e) {
                const unsigned lo = e & ((1u << lowrun) - 1u), top = e >> lowrun;
                return lo | (t << lowrun) | (top << g);
            };
            // tile t: run `top` (2^lowrun amplitudes at t << lowrun | top << g)
            // to sm[top << lowrun]
            auto load_tile = [&](const float2 *from, unsigned t) {
                if (run_bytes < 16) {  // runs below the bulk-copy granule: plain loads
                    for (unsigned e = threadIdx.x; e < GT; e += T) sm[e] = from[tile_index(t, e)];
                    __syncthreads();
                    return true;
                }
                before_copies();
                if (threadIdx.x == 0) mbar_expect_tx(s_bar, 8u * GT);
                __syncthreads();
                for (unsigned top = threadIdx.x; top < nchunks; top += T) {
                    bulk_copy(sm + (top << lowrun), from + ((size_t)t << lowrun) + ((size_t)top << g), run_bytes,
                              s_bar);
                }
                return wait_copies();
            };
            for (int l = 0; l < L && !failed; ++l) {
                const double *al = ang + 2 * l * n;
                layer_setup(al, n);
                build_phase_table(s_tlo, 7, s_ph, s_gph);
                build_phase_table(s_thi, g - 7, s_ph + 7, make_float2(1.f, 0.f));
                build_phase_table(s_ttop, h, s_ph + g, make_float2(1.f, 0.f));
                // the pair pass's rotations in kPairOrder; the top-qubit
                // pass's masks (tile bits lowrun..g)
                if (threadIdx.x < (unsigned)g) s_rotp[threadIdx.x] = s_rot[kPairOrder[threadIdx.x]];
                if (threadIdx.x < (unsigned)h) s_mask[g + threadIdx.x] = 1u << (lowrun + threadIdx.x);
                __syncthreads();
                // pair pass: src (through the pending permutation) -> dst, RY
                // on qubits 0..g-1 over both chunks at once, their RZ phases
                // on the way out
                for (unsigned pr = 0; pr < nchunks / 2 && !failed; ++pr) {
                    if (!load_pair(src, pr)) {
                        failed = true;
                        break;
                    }
                    if (permuted)
                        pair_gates<true>(sm, s_rotp);
                    else
                        pair_gates<false>(sm, s_rotp);
                    store_pair(dst, pr, true, s_flip & gmask);
                }
                // high pass on dst, in place: RY on the top qubits, then
                // their RZ phases on the way out
                for (unsigned t = 0; t < ntiles && !failed; ++t) {
                    if (!load_tile(dst, t)) {
                        failed = true;
                        break;
                    }
                    gates_blocked(sm, g + 1, s_mask + g, s_rot + g, h);
                    const unsigned fhi = s_flip >> g;  // flips of the top qubits
                    for (unsigned e = threadIdx.x; e < GT; e += T) {
                        const unsigned ef = e ^ (fhi << lowrun);
                        dst[tile_index(t, e)] = cmul(sm[ef], s_ttop[ef >> lowrun]);
                    }
                    __syncthreads();
                }
                float2 *tmp = src;
                src = dst;
                dst = tmp;
                permuted = true;  // this layer's CNOT ladder is still to be applied
            }
            // the last permutation, with the ZZ terms and the X terms of
            // qubits 0..g-1 read on the way; then the top qubits' X terms
            float zf = 0.f, xf = 0.f;
            for (unsigned pr = 0; pr < nchunks / 2 && !failed; ++pr) {
                if (!load_pair(src, pr)) {
                    failed = true;
                    break;
                }
                const unsigned hb = pr ^ hmask;
                for (unsigned e = threadIdx.x; e < 2 * G; e += T) {
                    const unsigned long long gi = ((unsigned long long)(e < G ? pr : hb) << g) | (e & gmask);
                    const float w = norm2(sm[pair_pos(e)]);
                    zf += w * (float)((n - 1) - 2 * __popcll((gi ^ (gi >> 1)) & ((1ull << (n - 1)) - 1ull)));
                }
                for (int q = 0; q < g; ++q) {
                    // logical pairs (e, e ^ 2^q) are the buffer pairs (p, p ^ (3 << q))
                    // (single bits if no layer ran: the buffer is in logical order);
                    // Re(conj(a) b) does not depend on which of the two is which
                    const unsigned msk = (permuted ? 3u : 1u) << q, low = (1u << q) - 1u;
                    for (unsigned u = threadIdx.x; u < G; u += T) {
                        const unsigned p0 = ((u & ~low) << 1) | (u & low);
                        const float2 a = sm[p0], b = sm[p0 ^ msk];
                        xf += 2.f * (a.x * b.x + a.y * b.y);
                    }
                }
                store_pair(dst, pr, false, 0u);
            }
            for (unsigned t = 0; t < ntiles && !failed; ++t) {
                if (!load_tile(dst, t)) {
                    failed = true;
                    break;
                }
                for (int q = g; q < n; ++q) xf += x_chunk(sm, g + 1, lowrun + (q - g));
                __syncthreads();
            }
            zz = (double)zf;
            xx = (double)xf;
            if (failed) break;  // the error flag is set; this CTA stops
        }
        const double zzs = block_sum_d(zz, s_red);
        const double xxs = block_sum_d(xx, s_red);
        if (threadIdx.x == 0) A.energies[c] = -zzs - A.h * xxs;
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side: the batch object, its graph and the tile autotuner
// ---------------------------------------------------------------------------
struct qsim_batch {
    int count = 0, nmax = 0, nmin = 0;
    long long nangles = 0;
    double h = 0.7;
    std::vector<int> nq, nl, order;
    std::vector<long long> aoff;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, sms = 0;
    // device memory
    unsigned char *mem = nullptr;
    size_t mem_bytes = 0;
    bool own_mem = false;
    double *d_angles = nullptr, *d_energies = nullptr;
    int *d_order = nullptr, *d_nq = nullptr, *d_nl = nullptr;
    long long *d_aoff = nullptr;
    unsigned int *d_counter = nullptr;
    float2 *d_gbuf = nullptr;
    size_t gstride = 0;
    int max_grid = 0;
    // pinned staging
    double *h_angles = nullptr, *h_energies = nullptr;
    unsigned int *h_flag = nullptr;  // the device error flag after a run
    // tuned launch configuration and its graph
    int threads = 512, m = 13, grid = 0;
    cudaGraphExec_t graph = nullptr;
    std::string err;
};

namespace {

constexpr int kCandidates[][2] = {{256, 12}, {256, 13}, {512, 12}, {512, 13}, {512, 14}, {1024, 13}, {1024, 14}};

int reg_amps(int threads) { return threads == 256 ? RegAmps<256>::value : threads == 512 ? RegAmps<512>::value
                                                                                       : RegAmps<1024>::value; }

typedef void (*VqeKernel)(const VqeArgs);
VqeKernel kernel_for(int threads) {
    return threads == 256 ? k_vqe_batch<256, false> : threads == 512 ? k_vqe_batch<512, false>
                                                                     : k_vqe_batch<1024, false>;
}

// The global-memory kernel: 256 threads, chunks of 2^12 amplitudes (a pair
// of them is 64 KB of shared memory, followed by the phase table of the top
// n - 12 qubits, 2 KB for n = 20, 32 KB for n = 24), two CTAs per SM
// (measured faster than three, which force the registers down to 80 and
// spill).
static_assert(kGlobalBits == 12, "kPairOrder lists the 12 chunk qubits");
constexpr int kMaxBatchQubits = 2 * kGlobalBits;  // n <= 2 g: a tile's runs are whole amplitudes
size_t global_smem(int nmax) {
    return ((size_t)16 << kGlobalBits) + ((size_t)8 << std::max(nmax - kGlobalBits, 0));
}
static_assert(kGlobalBits % 4 == 0, "pair-pass rotation groups must not need identity padding");

// circuits with more than m qubits: a prefix of the order (sorted by size)
int count_large(const qsim_batch *b, int m) {
    int k = 0;
    while (k < b->count && b->nq[b->order[k]] > m) ++k;
    return k;
}

bool config_valid(const qsim_batch *b, int threads, int m) {
    (void)b;
    return (1 << m) <= reg_amps(threads) * threads;  // in-place permutation through registers
}

int occupancy_global(const qsim_batch *b, int *grid) {
    VqeKernel k = k_vqe_batch<kGlobalThreads, true>;
    const size_t smem = global_smem(b->nmax);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return QSIM_ECUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kGlobalThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return QSIM_ENOTSUP;
    *grid = std::min(b->sms * per_sm, b->max_grid);
    return QSIM_OK;
}

int occupancy(const qsim_batch *b, int threads, int m, int *grid) {
    const size_t smem = (size_t)8 << m;
    VqeKernel k = kernel_for(threads);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return QSIM_ECUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess || per_sm < 1) return QSIM_ENOTSUP;
    *grid = std::min(b->sms * per_sm, b->max_grid);
    return QSIM_OK;
}

int berr(qsim_batch *b, int code, const std::string &msg) {
    b->err = msg;
    return code;
}

int launch(qsim_batch *b, int threads, int m, int grid) {
    const int large = count_large(b, m);
    // the two queues' counters and the error flag
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, 3 * sizeof(unsigned int), b->stream);
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    VqeArgs a;
    a.order = b->d_order;
    a.nq = b->d_nq;
    a.nl = b->d_nl;
    a.aoff = b->d_aoff;
    a.angles = b->d_angles;
    a.energies = b->d_energies;
    a.err = b->d_counter + 2;
    a.m = m;
    a.gbuf = b->d_gbuf;
    a.gstride = b->gstride;
    a.h = b->h;
    if (large > 0) {
        // the larger circuits first, several CTAs per SM
        int ggrid = 0;
        const int rc = occupancy_global(b, &ggrid);
        if (rc) return berr(b, rc, "occupancy query failed");
        a.counter = b->d_counter;
        a.begin = 0;
        a.end = large;
        k_vqe_batch<kGlobalThreads, true><<<ggrid, kGlobalThreads, global_smem(b->nmax), b->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    }
    if (large < b->count) {
        a.counter = b->d_counter + 1;
        a.begin = large;
        a.end = b->count;
        kernel_for(threads)<<<grid, threads, (size_t)8 << m, b->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    }
    return QSIM_OK;
}

// Capture angles H2D -> queue reset -> persistent kernel -> energies D2H.
int build_graph(qsim_batch *b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    int grid = 0;
    int rc = occupancy(b, b->threads, b->m, &grid);
    if (rc) return berr(b, rc, "occupancy query failed");
    b->grid = grid;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    cudaMemcpyAsync(b->d_angles, b->h_angles, sizeof(double) * b->nangles, cudaMemcpyHostToDevice, b->stream);
    rc = launch(b, b->threads, b->m, grid);
    cudaMemcpyAsync(b->h_energies, b->d_energies, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(b->h_flag, b->d_counter + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream);
    e = cudaStreamEndCapture(b->stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    return QSIM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int sim_batch_workspace_bytes(int count, const int *nqubits, const int *layers, size_t *bytes) {
    if (count < 1 || !nqubits || !layers || !bytes) return QSIM_EINVAL;
    long long nang = 0;
    int nmax = 0;
    for (int i = 0; i < count; ++i) {
        if (nqubits[i] < 2 || nqubits[i] > kMaxBatchQubits || layers[i] < 0) return QSIM_EINVAL;
        nang += 2LL * nqubits[i] * layers[i];
        nmax = std::max(nmax, nqubits[i]);
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return QSIM_ECUDA;
    }
    const size_t max_grid = (size_t)sms * 4;
    const size_t gstride = nmax > 12 ? ((size_t)1 << nmax) : 0;
    size_t s = align256(sizeof(double) * nang) + align256(sizeof(double) * count) + 3 * align256(sizeof(int) * count) +
               align256(sizeof(long long) * count) + 256 + max_grid * 2 * gstride * sizeof(float2);
    *bytes = s;
    return QSIM_OK;
}

int sim_batch_create(int count, const int *nqubits, const int *layers, double h, void *stream, void *workspace,
                     size_t workspace_bytes, qsim_batch **out) {
    if (!out) return QSIM_EINVAL;
    *out = nullptr;
    size_t need = 0;
    int rc = sim_batch_workspace_bytes(count, nqubits, layers, &need);
    if (rc) return rc;
    if (!std::isfinite(h)) return QSIM_ENONFINITE;
    qsim_batch *b = new (std::nothrow) qsim_batch();
    if (!b) return QSIM_ENOMEM;
    b->count = count;
    b->h = h;
    b->nq.assign(nqubits, nqubits + count);
    b->nl.assign(layers, layers + count);
    b->aoff.resize(count);
    long long off = 0;
    b->nmax = 0;
    b->nmin = 64;
    for (int i = 0; i < count; ++i) {
        b->aoff[i] = off;
        off += 2LL * nqubits[i] * layers[i];
        b->nmax = std::max(b->nmax, nqubits[i]);
        b->nmin = std::min(b->nmin, nqubits[i]);
    }
    b->nangles = off;
    // largest first: by qubits, then layers (so the circuits above any
    // shared-memory threshold m are a prefix of the order)
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return b->nq[x] != b->nq[y] ? b->nq[x] > b->nq[y] : b->nl[x] > b->nl[y];
    });
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->max_grid = b->sms * 4;
    b->gstride = b->nmax > 12 ? ((size_t)1 << b->nmax) : 0;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return QSIM_ECUDA;
        }
        b->own_stream = true;
    }
    if (workspace) {
        if (workspace_bytes < need || ((uintptr_t)workspace & 255u)) {
            sim_batch_destroy(b);
            return QSIM_EINVAL;
        }
        b->mem = (unsigned char *)workspace;
    } else {
        if (cudaMalloc((void **)&b->mem, need) != cudaSuccess) {
            cudaGetLastError();
            b->mem = nullptr;
            sim_batch_destroy(b);
            return QSIM_ENOMEM;
        }
        b->own_mem = true;
    }
    b->mem_bytes = need;
    unsigned char *p = b->mem;
    b->d_angles = (double *)p;
    p += align256(sizeof(double) * b->nangles);
    b->d_energies = (double *)p;
    p += align256(sizeof(double) * count);
    b->d_order = (int *)p;
    p += align256(sizeof(int) * count);
    b->d_nq = (int *)p;
    p += align256(sizeof(int) * count);
    b->d_nl = (int *)p;
    p += align256(sizeof(int) * count);
    b->d_aoff = (long long *)p;
    p += align256(sizeof(long long) * count);
    b->d_counter = (unsigned int *)p;
    p += 256;
    b->d_gbuf = (float2 *)p;
    if (cudaMallocHost((void **)&b->h_angles, sizeof(double) * std::max<long long>(1, b->nangles)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_energies, sizeof(double) * count) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_flag, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        sim_batch_destroy(b);
        return QSIM_ENOMEM;
    }
    cudaMemcpyAsync(b->d_order, b->order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_nq, b->nq.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_nl, b->nl.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_aoff, b->aoff.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, b->stream);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        sim_batch_destroy(b);
        return QSIM_ECUDA;
    }
    // default configuration: the largest valid shared-memory threshold
    b->threads = 512;
    b->m = 0;
    for (int m = 14; m >= 12; --m)
        if (config_valid(b, 512, m)) {
            b->m = m;
            break;
        }
    if (!b->m) {
        sim_batch_destroy(b);
        return QSIM_ENOTSUP;
    }
    *out = b;
    return QSIM_OK;
}

int sim_batch_destroy(qsim_batch *b) {
    if (!b) return QSIM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->own_mem && b->mem) cudaFree(b->mem);
    if (b->h_angles) cudaFreeHost(b->h_angles);
    if (b->h_energies) cudaFreeHost(b->h_energies);
    if (b->h_flag) cudaFreeHost(b->h_flag);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return QSIM_OK;
}

int sim_batch_run(qsim_batch *b, const double *angles, double *energies) {
    if (!b || (!angles && b->nangles) || !energies) return QSIM_EINVAL;
    for (long long i = 0; i < b->nangles; ++i)
        if (!std::isfinite(angles[i])) return berr(b, QSIM_ENONFINITE, "non-finite angle");
    if (!b->graph) {
        int rc = build_graph(b);
        if (rc) return rc;
    }
    std::memcpy(b->h_angles, angles, sizeof(double) * b->nangles);
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    if (*b->h_flag) return berr(b, QSIM_ETIMEOUT, "a bounded wait for bulk copies gave up; energies not computed");
    std::memcpy(energies, b->h_energies, sizeof(double) * b->count);
    return QSIM_OK;
}

int sim_batch_autotune(qsim_batch *b, const double *angles, int reps, int *threads_out, int *m_out) {
    if (!b || (!angles && b->nangles) || reps < 1) return QSIM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(b->d_angles, angles, sizeof(double) * b->nangles, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bt = b->threads, bm = b->m;
    for (const auto &cand : kCandidates) {
        const int threads = cand[0], m = cand[1];
        if (!config_valid(b, threads, m)) continue;
        int grid = 0;
        if (occupancy(b, threads, m, &grid)) continue;
        std::vector<float> t;
        for (int r = 0; r <= reps; ++r) {
            cudaEventRecord(e0, b->stream);
            int rc = launch(b, threads, m, grid);
            cudaEventRecord(e1, b->stream);
            if (rc) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) t.push_back(ms);  // first run is a warm-up
        }
        if ((int)t.size() != reps) continue;
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (med < best) {
            best = med;
            bt = threads;
            bm = m;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(b, QSIM_ECUDA, cudaGetErrorString(e));
    b->threads = bt;
    b->m = bm;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (threads_out) *threads_out = bt;
    if (m_out) *m_out = bm;
    return QSIM_OK;
}

int sim_batch_set_config(qsim_batch *b, int threads, int m) {
    if (!b) return QSIM_EINVAL;
    if (threads != 256 && threads != 512 && threads != 1024) return berr(b, QSIM_EINVAL, "threads must be 256/512/1024");
    if (m < 12 || m > 14 || !config_valid(b, threads, m)) return berr(b, QSIM_EINVAL, "invalid tile configuration");
    b->threads = threads;
    b->m = m;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return QSIM_OK;
}

const char *sim_batch_last_error(const qsim_batch *b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"

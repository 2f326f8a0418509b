// diag_kernels.cu -- a block of diagonal gates applied in one pass.
//
// Gates whose matrices are diagonal (Z, S, T, R(phi), RZ, CZ, controlled
// phases, multi-controlled Z) only multiply each amplitude by a phase that
// depends on the bits of its index on the gate's qubits, and they commute
// with one another.  A run of them over a qubit set S (|S| <= 12) is one
// table d of 2^|S| factors (built on the host in FP64: the product of the
// gates' diagonal entries for every assignment of S), and the pass is
//     psi_i <- d[bits of i on S] * psi_i.
// The phase ladders of the QFT (ProjectQ paper, Sec. 3: the constant adder
// is QFT, phase shifts, inverse QFT) and the controlled z-rotation chain of
// the simulator benchmark (Sec. 4.3.2, Fig. 7) are made of such gates.
//
// The table and five 256-entry bit-gather tables (index bits 0..39 -> bits
// of the table index) are copied to shared memory per CTA.  A CTA takes
// contiguous chunks of up to 2^16 amplitudes, so the table-index bits of
// index bits 16 and above are gathered once per chunk; each thread handles
// 16 bytes of amplitudes per access (two complex64 or one complex128),
// eight accesses in flight.
// complex128 uses FP64 products, or double-float products when the handle
// runs complex128 gates in double-float arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "df128.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kDiagThreads = 256;

template <typename Amp>
__global__ void __launch_bounds__(kDiagThreads) k_diag_block(Amp *__restrict__ psi, uint64_t nchunks, int cb, int k,
                                                            const unsigned char *__restrict__ rec, int use_df) {
    extern __shared__ unsigned char sm_raw[];
    Amp *d = (Amp *)sm_raw;
    uint16_t *gather = (uint16_t *)(sm_raw + (sizeof(Amp) << k));  // [5][256]
    const int D = 1 << k;
    const Amp *gd = (const Amp *)rec;
    const uint16_t *gg = (const uint16_t *)(rec + (sizeof(Amp) << k));
    for (int i = threadIdx.x; i < D; i += blockDim.x) d[i] = gd[i];
    for (int i = threadIdx.x; i < 5 * 256; i += blockDim.x) gather[i] = gg[i];
    __syncthreads();
    constexpr int kU = 8;                    // 16-byte accesses in flight per thread
    constexpr int kPer = 16 / sizeof(Amp);   // amplitudes per access
    const unsigned units = (1u << cb) / kPer;  // accesses per chunk
    for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const uint64_t base = ch << cb;
        // table-index bits of index bits 16.. (constant over the chunk, cb <= 16)
        const unsigned hi = (unsigned)gather[512 + ((base >> 16) & 255)] | gather[768 + ((base >> 24) & 255)] |
                            gather[1024 + ((base >> 32) & 255)];
        const unsigned lo0 = (unsigned)(base & 0xFFFFu);
        auto tidx = [&](unsigned idx) {
            const unsigned lo = lo0 | (idx * kPer);
            return (unsigned)gather[lo & 255] | gather[256 + (lo >> 8)] | hi;
        };
        for (unsigned u0 = threadIdx.x; u0 < units; u0 += kU * kDiagThreads) {
            if (sizeof(Amp) == 8) {
                // two complex64 per access; the second's table index adds
                // index bit 0 to the first's
                float4 *p4 = (float4 *)psi + (base >> 1);
                const float2 *df = (const float2 *)d;
                const unsigned bit0 = gather[1];
                float4 v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (u0 + u * kDiagThreads < units) v[u] = p4[u0 + u * kDiagThreads];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const unsigned idx = u0 + u * kDiagThreads;
                    if (idx >= units) continue;
                    const unsigned t0 = tidx(idx);
                    const float2 a = cmul(df[t0], make_float2(v[u].x, v[u].y));
                    const float2 b = cmul(df[t0 | bit0], make_float2(v[u].z, v[u].w));
                    p4[idx] = make_float4(a.x, a.y, b.x, b.y);
                }
            } else {
                double2 *p2 = (double2 *)psi + base;
                const double2 *dd = (const double2 *)d;
                double2 v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (u0 + u * kDiagThreads < units) v[u] = p2[u0 + u * kDiagThreads];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const unsigned idx = u0 + u * kDiagThreads;
                    if (idx >= units) continue;
                    const double2 z = dd[tidx(idx)];
                    if (use_df) {
                        const qsim_df::C2 w = qsim_df::split(z);
                        p2[idx] = qsim_df::to_double(qsim_df::cmul(w, qsim_df::split(v[u])));
                    } else {
                        p2[idx] = cmul(z, v[u]);
                    }
                }
            }
        }
    }
}

template <typename Amp> Amp to_amp(cd z);
template <> double2 to_amp<double2>(cd z) { return make_double2(z.real(), z.imag()); }
template <> float2 to_amp<float2>(cd z) { return make_float2((float)z.real(), (float)z.imag()); }

template <typename Amp>
int diag_block(qsim *s, uint64_t dmask, const cd *dt) {
    const int k = __builtin_popcountll(dmask);
    if (k < 1 || k > kMaxDiagQubits) return set_err(s, QSIM_EINVAL, "diagonal block width");
    // record: table (2^k Amp) then 5 x 256 uint16 gather tables
    const size_t tbytes = sizeof(Amp) << k, gbytes = 5 * 256 * sizeof(uint16_t);
    std::vector<unsigned char> rec(tbytes + gbytes);
    std::vector<Amp> tab(1u << k);
    for (int r = 0; r < (1 << k); ++r) tab[r] = to_amp<Amp>(dt[r]);
    std::memcpy(rec.data(), tab.data(), tbytes);
    int pos[64], np = 0;
    for (int b = 0; b < 64; ++b)
        if ((dmask >> b) & 1ull) pos[b] = np++;
        else pos[b] = -1;
    std::vector<uint16_t> g(5 * 256, 0);
    for (int c = 0; c < 5; ++c)
        for (int v = 0; v < 256; ++v) {
            uint16_t r = 0;
            for (int bit = 0; bit < 8; ++bit)
                if ((v >> bit) & 1) {
                    const int b = 8 * c + bit;
                    if (b < 64 && pos[b] >= 0) r |= (uint16_t)(1u << pos[b]);
                }
            g[c * 256 + v] = r;
        }
    std::memcpy(rec.data() + tbytes, g.data(), gbytes);
    unsigned char *dev = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev);
    if (rc) return rc;
    const size_t smem = tbytes + gbytes;
    static bool attr[2][64] = {{false}};
    const int which = sizeof(Amp) == 8 ? 0 : 1;
    if (s->device >= 0 && s->device < 64 && !attr[which][s->device]) {
        cudaError_t e = cudaFuncSetAttribute(k_diag_block<Amp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((sizeof(Amp) << kMaxDiagQubits) + gbytes));
        if (e != cudaSuccess) return cuda_err(s, e, "diagonal kernel attribute");
        attr[which][s->device] = true;
    }
    // contiguous chunks of 2^cb amplitudes (cb <= 16), at least about four
    // per SM where the register allows
    const int n = s->n;
    const int cb = std::max(std::min(n, 9), std::min(16, n - 10));
    const uint64_t nchunks = 1ull << (n - cb);
    const uint64_t grid = nchunks < (uint64_t)s->sms * 8 ? nchunks : (uint64_t)s->sms * 8;
    k_diag_block<Amp><<<(unsigned)grid, kDiagThreads, smem, s->stream>>>((Amp *)s->state, nchunks, cb, k, dev,
                                                                           s->c128_df ? 1 : 0);
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "diagonal block launch");
}

}  // namespace

int launch_block_diag(qsim *s, uint64_t dmask, const cd *d) {
    if (s->n < 2) return set_err(s, QSIM_ENOTSUP, "diagonal block needs n >= 2");
    return s->prec == QSIM_C128 ? diag_block<double2>(s, dmask, d) : diag_block<float2>(s, dmask, d);
}

// perm_kernels.cu -- emulation of a classical reversible function on a
// register: |..., x, ...> -> |..., f(x), ...> for a bijection f on the 2^m
// values of an m-qubit register, where all control qubits are |1>.
//
// The paper's emulator applies classical functions to a superposition
// directly instead of simulating the gates that compute them (ProjectQ
// paper, Sec. 4.3.3: BasicMathGate, e.g. AddConstant(c): x -> x + c; the
// modular multiplication of Shor's algorithm, Appendix A.3).  A bijection
// only moves amplitudes: for every group of the 2^m amplitudes that share
// the bits outside the register (and have all controls set), the amplitude
// at register value x moves to register value f(x).
//
// A CTA works on tiles of 2^m register values x 2^c runs: the c lowest
// qubits outside the register and the controls, chosen so that a tile holds
// 2^13 amplitudes (or all of the register's 2^m) and a run at least 32
// bytes (one DRAM sector) where such qubits exist.
// f acts on every run alike, so a tile maps onto
// itself: the CTA loads it into shared memory (16 loads per thread in flight
// for complex64, 8 for complex128), the index holding the lowest address bit
// varying fastest so that the loads are coalesced whether the register holds
// the low qubits or the high ones; it synchronises, and writes each position
// from its source, out(v, r) = in(f^-1(v), r), so the stores are coalesced
// too.  The register-value and run offsets and f^-1 come from a device
// record (uint64 offsets, uint32 values) and are copied to shared memory
// once per CTA.  m <= 12.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kPermThreads = 256;
constexpr size_t kPermSmemMax = 128u << 10;  // a tile's amplitudes in shared memory (plus the tables)

// tile element e <-> (register value v, run r); v_fast: e = r * 2^m + v,
// else e = v * 2^c + r
__device__ __forceinline__ void split_e(unsigned e, int m, int c, bool v_fast, unsigned &v, unsigned &r) {
    if (v_fast) {
        v = e & ((1u << m) - 1u);
        r = e >> m;
    } else {
        v = e >> c;
        r = e & ((1u << c) - 1u);
    }
}

template <typename Amp>
__global__ void __launch_bounds__(kPermThreads) k_permute(Amp *__restrict__ psi, uint64_t ntiles, const InsertSpec ins,
                                                          uint64_t cmask, int m, int c, int v_fast,
                                                          const uint64_t *__restrict__ goff,
                                                          const uint64_t *__restrict__ groff,
                                                          const uint32_t *__restrict__ gfinv) {
    // shared memory: the tile, then the tables (offsets of register values
    // and runs, f^-1), copied once per CTA
    extern __shared__ unsigned char sm_raw[];
    Amp *buf = (Amp *)sm_raw;
    const unsigned T = 1u << (m + c), D = 1u << m, R = 1u << c;
    uint64_t *off = (uint64_t *)(sm_raw + sizeof(Amp) * T);
    uint64_t *roff = off + D;
    uint32_t *finv = (uint32_t *)(roff + R);
    for (unsigned i = threadIdx.x; i < D; i += kPermThreads) {
        off[i] = goff[i];
        finv[i] = gfinv[i];
    }
    for (unsigned i = threadIdx.x; i < R; i += kPermThreads) roff[i] = groff[i];
    __syncthreads();
    constexpr int kL = sizeof(Amp) == 8 ? 16 : 8;  // loads in flight per thread per round
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t base = insert_zeros(t, ins) | cmask;
        for (unsigned e0 = threadIdx.x; e0 < T; e0 += kL * kPermThreads) {
            Amp a[kL];
#pragma unroll
            for (int u = 0; u < kL; ++u) {
                const unsigned e = e0 + u * kPermThreads;
                if (e < T) {
                    unsigned v, r;
                    split_e(e, m, c, v_fast, v, r);
                    a[u] = psi[base + off[v] + roff[r]];
                }
            }
#pragma unroll
            for (int u = 0; u < kL; ++u) {
                const unsigned e = e0 + u * kPermThreads;
                if (e < T) buf[e] = a[u];
            }
        }
        __syncthreads();
        for (unsigned e = threadIdx.x; e < T; e += kPermThreads) {
            unsigned v, r;
            split_e(e, m, c, v_fast, v, r);
            const unsigned fv = finv[v];
            psi[base + off[v] + roff[r]] = buf[v_fast ? ((r << m) | fv) : ((fv << c) | r)];
        }
        __syncthreads();
    }
}

template <typename Amp>
int permute(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask) {
    const int D = 1 << m;
    const int n = s->n;
    // run qubits: the lowest outside the register and the controls
    const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    const uint64_t free = all & ~(qmask | cmask);
    const int cmin = sizeof(Amp) == 8 ? 2 : 1;  // runs of at least 32 bytes
    int c = 13 - m < cmin ? cmin : 13 - m;      // tiles of 2^13 amplitudes
    while (c > 0 && ((size_t)sizeof(Amp) << (m + c)) > kPermSmemMax) --c;
    if (c > __builtin_popcountll(free)) c = __builtin_popcountll(free);
    int rbit[64], nr = 0;
    for (int b = 0; b < n && nr < c; ++b)
        if ((free >> b) & 1ull) rbit[nr++] = b;
    uint64_t rmask = 0;
    for (int j = 0; j < c; ++j) rmask |= 1ull << rbit[j];
    const int R = 1 << c;
    std::vector<unsigned char> rec(sizeof(uint64_t) * (D + R) + sizeof(uint32_t) * D);
    uint64_t *off = (uint64_t *)rec.data();
    uint64_t *roff = off + D;
    uint32_t *finv = (uint32_t *)(rec.data() + sizeof(uint64_t) * (D + R));
    for (int v = 0; v < D; ++v) {
        uint64_t a = 0;
        for (int j = 0; j < m; ++j)
            if ((v >> j) & 1) a |= 1ull << qubits[j];
        off[v] = a;
        finv[perm[v]] = (uint32_t)v;
    }
    for (int r = 0; r < R; ++r) {
        uint64_t a = 0;
        for (int j = 0; j < c; ++j)
            if ((r >> j) & 1) a |= 1ull << rbit[j];
        roff[r] = a;
    }
    // the index holding the lowest address bit varies fastest
    const uint64_t low = (qmask | rmask) & (0ull - (qmask | rmask));
    const int v_fast = (low & qmask) ? 1 : 0;
    unsigned char *dev = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev);
    if (rc) return rc;
    InsertSpec ins{};
    ins.m = 0;
    const uint64_t fixed = qmask | cmask | rmask;
    for (int b = 0; b < 64; ++b)
        if ((fixed >> b) & 1ull) ins.pos[ins.m++] = b;
    const uint64_t ntiles = 1ull << (n - ins.m);
    const size_t smem = (sizeof(Amp) << (m + c)) + sizeof(uint64_t) * (D + R) + sizeof(uint32_t) * D;
    static bool attr[2][64] = {{false}};
    const int which = sizeof(Amp) == 8 ? 0 : 1;
    if (s->device >= 0 && s->device < 64 && !attr[which][s->device]) {
        cudaError_t e = cudaFuncSetAttribute(k_permute<Amp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kPermSmemMax + (size_t)12 * 4096 + 8 * 4096));
        if (e != cudaSuccess) return cuda_err(s, e, "permutation kernel attribute");
        attr[which][s->device] = true;
    }
    const uint64_t grid = ntiles < (uint64_t)kSMs * 8 ? ntiles : (uint64_t)kSMs * 8;
    k_permute<Amp><<<(unsigned)grid, kPermThreads, smem, s->stream>>>(
        (Amp *)s->state, ntiles, ins, cmask, m, c, v_fast, (const uint64_t *)dev, (const uint64_t *)dev + D,
        (const uint32_t *)(dev + sizeof(uint64_t) * (D + R)));
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "permutation launch");
}

}  // namespace

int launch_permutation(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask) {
    return s->prec == QSIM_C128 ? permute<double2>(s, perm, qubits, m, qmask, cmask)
                                : permute<float2>(s, perm, qubits, m, qmask, cmask);
}

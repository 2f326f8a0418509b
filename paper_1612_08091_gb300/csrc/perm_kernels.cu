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
// Each CTA takes groups in turn: it gathers the group into shared memory,
// synchronises, and scatters every amplitude to its new position.  The
// register-value -> address offsets and f are read from a device record
// (uint64 offsets, uint32 values).  m <= 12.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

constexpr int kPermThreads = 256;

template <typename Amp>
__global__ void __launch_bounds__(kPermThreads) k_permute(Amp *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                          uint64_t cmask, int m, const uint64_t *__restrict__ off,
                                                          const uint32_t *__restrict__ f) {
    extern __shared__ unsigned char sm_raw[];
    Amp *buf = (Amp *)sm_raw;
    const int D = 1 << m;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const uint64_t base = insert_zeros(g, ins) | cmask;
        for (int v = threadIdx.x; v < D; v += blockDim.x) buf[v] = psi[base + off[v]];
        __syncthreads();
        for (int v = threadIdx.x; v < D; v += blockDim.x) psi[base + off[f[v]]] = buf[v];
        __syncthreads();
    }
}

template <typename Amp>
int permute(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask) {
    const int D = 1 << m;
    std::vector<unsigned char> rec(sizeof(uint64_t) * D + sizeof(uint32_t) * D);
    uint64_t *off = (uint64_t *)rec.data();
    uint32_t *f = (uint32_t *)(rec.data() + sizeof(uint64_t) * D);
    for (int v = 0; v < D; ++v) {
        uint64_t a = 0;
        for (int j = 0; j < m; ++j)
            if ((v >> j) & 1) a |= 1ull << qubits[j];
        off[v] = a;
        f[v] = (uint32_t)perm[v];
    }
    unsigned char *dev = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev);
    if (rc) return rc;
    InsertSpec ins{};
    ins.m = 0;
    const uint64_t fixed = qmask | cmask;
    for (int b = 0; b < 64; ++b)
        if ((fixed >> b) & 1ull) ins.pos[ins.m++] = b;
    const uint64_t ngroups = 1ull << (s->n - ins.m);
    const size_t smem = sizeof(Amp) * D;
    static bool attr[2][64] = {{false}};
    const int which = sizeof(Amp) == 8 ? 0 : 1;
    if (s->device >= 0 && s->device < 64 && !attr[which][s->device]) {
        cudaError_t e = cudaFuncSetAttribute(k_permute<Amp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(Amp) << 12));
        if (e != cudaSuccess) return cuda_err(s, e, "permutation kernel attribute");
        attr[which][s->device] = true;
    }
    const uint64_t grid = ngroups < (uint64_t)kSMs * 8 ? ngroups : (uint64_t)kSMs * 8;
    k_permute<Amp><<<(unsigned)grid, kPermThreads, smem, s->stream>>>(
        (Amp *)s->state, ngroups, ins, cmask, m, (const uint64_t *)dev,
        (const uint32_t *)(dev + sizeof(uint64_t) * D));
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "permutation launch");
}

}  // namespace

int launch_permutation(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask) {
    return s->prec == QSIM_C128 ? permute<double2>(s, perm, qubits, m, qmask, cmask)
                                : permute<float2>(s, perm, qubits, m, qmask, cmask);
}

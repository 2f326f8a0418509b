// gate_kernels.cu -- unfused ("plain") gate application, one launch per gate.
//
// The operation is the simulator's per-gate sweep over the 2^n amplitudes
// (ProjectQ paper, Sec. 4.3.2): for every group of amplitudes that differ
// only in the target bits and have every control bit equal to 1 (Sec. 4.1.3,
// Control), replace the 2^t amplitudes of the group by U times them.  Groups
// are enumerated directly by inserting zero bits at the target and control
// positions into a group counter, so a gate with c controls touches only the
// 2^(n-c) amplitudes it changes (a 27-control Z on 28 qubits touches 2).
//
// Each thread owns one group: it gathers 2^t amplitudes, multiplies, and
// scatters.  complex128 uses FP64 arithmetic, complex64 FP32.  Specialised
// kernels avoid arithmetic the gate does not need: a phase on the all-ones
// subspace (Z, S, T, R(phi), CZ, multi-controlled Z), a diagonal one-qubit
// gate (RZ), and the X permutation (X, CNOT, Toffoli).
#include <algorithm>

#include "common.cuh"
#include "df128.cuh"
#include "internal.h"

using namespace qsim_dev;

namespace {

template <typename Amp> struct Mat1 { Amp m[4]; };
template <typename Amp, int K> struct MatK { Amp m[(1 << K) * (1 << K)]; uint64_t off[1 << K]; };

// One-qubit, phase and X kernels: each thread takes kGroups groups, g =
// block * 256 kGroups + u * 256 + thread (u < kGroups), and issues all their
// loads before any arithmetic, so that 4 to 8 amplitudes per thread are in
// flight (one group per thread left too few bytes in flight for HBM).
constexpr int kGroups = 4;
constexpr int kPhaseGroups = 8;  // the phase kernel loads one amplitude per group

inline unsigned blocks_for(uint64_t work, int threads) {
    return (unsigned)((work + (uint64_t)threads - 1) / (uint64_t)threads);
}

template <typename Amp>
__global__ void __launch_bounds__(256) k_dense1(Amp *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                uint64_t cmask, uint64_t tbit, const Mat1<Amp> M) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kGroups) + threadIdx.x;
    uint64_t i0[kGroups];
    Amp a[kGroups], b[kGroups];
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i0[u] = insert_zeros(g0 + u * 256, ins) | cmask;
            a[u] = psi[i0[u]];
            b[u] = psi[i0[u] | tbit];
        }
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            Amp na = cmul(M.m[0], a[u]);
            na = cfma(M.m[1], b[u], na);
            Amp nb = cmul(M.m[2], a[u]);
            nb = cfma(M.m[3], b[u], nb);
            psi[i0[u]] = na;
            psi[i0[u] | tbit] = nb;
        }
}

template <typename Amp, int K>
__global__ void __launch_bounds__(128) k_denseK(Amp *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                uint64_t cmask, const MatK<Amp, K> M) {
    constexpr int D = 1 << K;
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const uint64_t base = insert_zeros(g, ins) | cmask;
    Amp v[D];
#pragma unroll
    for (int r = 0; r < D; ++r) v[r] = psi[base + M.off[r]];
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
        Amp acc = cmul(M.m[r * D], v[0]);
#pragma unroll
        for (int c = 1; c < D; ++c) acc = cfma(M.m[r * D + c], v[c], acc);
        psi[base + M.off[r]] = acc;
    }
}

template <typename Amp>
__global__ void __launch_bounds__(256) k_phase(Amp *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                               uint64_t mask, Amp z) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kPhaseGroups) + threadIdx.x;
    uint64_t i[kPhaseGroups];
    Amp v[kPhaseGroups];
#pragma unroll
    for (int u = 0; u < kPhaseGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i[u] = insert_zeros(g0 + u * 256, ins) | mask;
            v[u] = psi[i[u]];
        }
#pragma unroll
    for (int u = 0; u < kPhaseGroups; ++u)
        if (g0 + u * 256 < ngroups) psi[i[u]] = cmul(z, v[u]);
}

template <typename Amp>
__global__ void __launch_bounds__(256) k_diag1(Amp *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                               uint64_t cmask, uint64_t tbit, Amp d0, Amp d1) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kGroups) + threadIdx.x;
    uint64_t i0[kGroups];
    Amp a[kGroups], b[kGroups];
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i0[u] = insert_zeros(g0 + u * 256, ins) | cmask;
            a[u] = psi[i0[u]];
            b[u] = psi[i0[u] | tbit];
        }
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            psi[i0[u]] = cmul(d0, a[u]);
            psi[i0[u] | tbit] = cmul(d1, b[u]);
        }
}

template <typename Amp>
__global__ void __launch_bounds__(256) k_x(Amp *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                           uint64_t cmask, uint64_t tbit) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kGroups) + threadIdx.x;
    uint64_t i0[kGroups];
    Amp a[kGroups], b[kGroups];
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i0[u] = insert_zeros(g0 + u * 256, ins) | cmask;
            a[u] = psi[i0[u]];
            b[u] = psi[i0[u] | tbit];
        }
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            psi[i0[u]] = b[u];
            psi[i0[u] | tbit] = a[u];
        }
}

// complex128 with double-float arithmetic (df128.cuh): one-qubit dense,
// diagonal and phase gates, kGroups (kPhaseGroups) groups per thread
struct MatDF {
    qsim_df::C2 m[4];
};

__global__ void __launch_bounds__(256) k_dense1_df(double2 *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                   uint64_t cmask, uint64_t tbit, const MatDF M) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kGroups) + threadIdx.x;
    uint64_t i0[kGroups];
    double2 a[kGroups], b[kGroups];
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i0[u] = insert_zeros(g0 + u * 256, ins) | cmask;
            a[u] = psi[i0[u]];
            b[u] = psi[i0[u] | tbit];
        }
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            const qsim_df::C2 x = qsim_df::split(a[u]), y = qsim_df::split(b[u]);
            psi[i0[u]] = qsim_df::to_double(qsim_df::cdot2(M.m[0], x, M.m[1], y));
            psi[i0[u] | tbit] = qsim_df::to_double(qsim_df::cdot2(M.m[2], x, M.m[3], y));
        }
}

__global__ void __launch_bounds__(256) k_diag1_df(double2 *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                  uint64_t cmask, uint64_t tbit, const MatDF M) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kGroups) + threadIdx.x;
    uint64_t i0[kGroups];
    double2 a[kGroups], b[kGroups];
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i0[u] = insert_zeros(g0 + u * 256, ins) | cmask;
            a[u] = psi[i0[u]];
            b[u] = psi[i0[u] | tbit];
        }
#pragma unroll
    for (int u = 0; u < kGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            psi[i0[u]] = qsim_df::to_double(qsim_df::cmul(M.m[0], qsim_df::split(a[u])));
            psi[i0[u] | tbit] = qsim_df::to_double(qsim_df::cmul(M.m[3], qsim_df::split(b[u])));
        }
}

__global__ void __launch_bounds__(256) k_phase_df(double2 *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                  uint64_t mask, const MatDF M) {
    const uint64_t g0 = blockIdx.x * (uint64_t)(256 * kPhaseGroups) + threadIdx.x;
    uint64_t i[kPhaseGroups];
    double2 v[kPhaseGroups];
#pragma unroll
    for (int u = 0; u < kPhaseGroups; ++u)
        if (g0 + u * 256 < ngroups) {
            i[u] = insert_zeros(g0 + u * 256, ins) | mask;
            v[u] = psi[i[u]];
        }
#pragma unroll
    for (int u = 0; u < kPhaseGroups; ++u)
        if (g0 + u * 256 < ngroups) psi[i[u]] = qsim_df::to_double(qsim_df::cmul(M.m[3], qsim_df::split(v[u])));
}

// complex128 k-qubit dense gate or fused block in double-float arithmetic:
// the group's 2^k amplitudes split into FP32 pairs, each output the sum of
// 2^k exact-product complex MACs with two-sum additions, rounded once to
// double.  About 40 FP32 operations per MAC instead of 4 FP64 FMAs (FP64
// runs at 1/58 of the FP32 rate here).
template <int K> struct MatKDF { qsim_df::C2 m[(1 << K) * (1 << K)]; uint64_t off[1 << K]; };

template <int K>
__global__ void __launch_bounds__(128) k_denseK_df(double2 *__restrict__ psi, uint64_t ngroups, const InsertSpec ins,
                                                   uint64_t cmask, const MatKDF<K> M) {
    constexpr int D = 1 << K;
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const uint64_t base = insert_zeros(g, ins) | cmask;
    qsim_df::C2 v[D];
#pragma unroll
    for (int r = 0; r < D; ++r) v[r] = qsim_df::split(psi[base + M.off[r]]);
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
        qsim_df::C2 acc = qsim_df::cmul(M.m[r * D], v[0]);
#pragma unroll
        for (int c = 1; c < D; ++c) acc = qsim_df::cadd(acc, qsim_df::cmul(M.m[r * D + c], v[c]));
        psi[base + M.off[r]] = qsim_df::to_double(acc);
    }
}

qsim_df::F2 host_split(double x) {
    qsim_df::F2 r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

MatDF make_df(const cd *m, int count) {
    MatDF M{};
    for (int i = 0; i < count; ++i) M.m[i] = qsim_df::C2{host_split(m[i].real()), host_split(m[i].imag())};
    return M;
}

// Returns true if the gate was launched on a double-float kernel.
bool gate_df(qsim *s, const GateRec &g) {
    if (g.t != 1) return false;
    double2 *psi = (double2 *)s->state;
    const uint64_t tbit = 1ull << g.targets[0];
    InsertSpec ins{};
    auto spec = [&](uint64_t mask) {
        ins.m = 0;
        for (int b = 0; b < 64; ++b)
            if ((mask >> b) & 1ull) ins.pos[ins.m++] = b;
    };
    const MatDF M = make_df(g.m.data(), 4);
    switch (g.kind) {
    case GK_DENSE: {
        spec(g.tmask | g.cmask);
        const uint64_t ng = 1ull << (s->n - ins.m);
        k_dense1_df<<<blocks_for(ng, 256 * kGroups), 256, 0, s->stream>>>(psi, ng, ins, g.cmask, tbit, M);
        return true;
    }
    case GK_DIAG1: {
        spec(g.tmask | g.cmask);
        const uint64_t ng = 1ull << (s->n - ins.m);
        k_diag1_df<<<blocks_for(ng, 256 * kGroups), 256, 0, s->stream>>>(psi, ng, ins, g.cmask, tbit, M);
        return true;
    }
    case GK_PHASE: {
        const uint64_t mask = g.tmask | g.cmask;
        spec(mask);
        const uint64_t ng = 1ull << (s->n - ins.m);
        k_phase_df<<<blocks_for(ng, 256 * kPhaseGroups), 256, 0, s->stream>>>(psi, ng, ins, mask, M);
        return true;
    }
    default:
        return false;
    }
}

InsertSpec make_spec(uint64_t mask) {
    InsertSpec s{};
    s.m = 0;
    for (int b = 0; b < 64; ++b)
        if ((mask >> b) & 1ull) s.pos[s.m++] = b;
    return s;
}

inline double2 to_amp(cd z, double2 *) { return make_double2(z.real(), z.imag()); }
inline float2 to_amp(cd z, float2 *) { return make_float2((float)z.real(), (float)z.imag()); }
template <typename Amp> Amp amp(cd z) { return to_amp(z, (Amp *)nullptr); }

template <int K>
int dense_k_df(qsim *s, const int *targets, uint64_t cmask, const cd *m) {
    constexpr int D = 1 << K;
    MatKDF<K> M;
    uint64_t tmask = 0;
    for (int j = 0; j < K; ++j) tmask |= 1ull << targets[j];
    for (int r = 0; r < D; ++r) {
        uint64_t o = 0;
        for (int j = 0; j < K; ++j)
            if ((r >> j) & 1) o |= 1ull << targets[j];
        M.off[r] = o;
    }
    for (int i = 0; i < D * D; ++i) M.m[i] = qsim_df::C2{host_split(m[i].real()), host_split(m[i].imag())};
    const InsertSpec ins = make_spec(tmask | cmask);
    const uint64_t ngroups = 1ull << (s->n - ins.m);
    k_denseK_df<K><<<blocks_for(ngroups, 128), 128, 0, s->stream>>>((double2 *)s->state, ngroups, ins, cmask, M);
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "double-float dense gate launch");
}

template <typename Amp, int K>
int dense_k(qsim *s, const int *targets, uint64_t cmask, const cd *m) {
    if constexpr (sizeof(Amp) == 16) {
        if (s->c128_df) return dense_k_df<K>(s, targets, cmask, m);
    }
    constexpr int D = 1 << K;
    MatK<Amp, K> M;
    uint64_t tmask = 0;
    for (int j = 0; j < K; ++j) tmask |= 1ull << targets[j];
    for (int r = 0; r < D; ++r) {
        uint64_t o = 0;
        for (int j = 0; j < K; ++j)
            if ((r >> j) & 1) o |= 1ull << targets[j];
        M.off[r] = o;
    }
    for (int i = 0; i < D * D; ++i) M.m[i] = amp<Amp>(m[i]);
    const InsertSpec ins = make_spec(tmask | cmask);
    const uint64_t ngroups = 1ull << (s->n - ins.m);
    k_denseK<Amp, K><<<blocks_for(ngroups, 128), 128, 0, s->stream>>>((Amp *)s->state, ngroups, ins, cmask, M);
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "dense gate launch");
}

template <typename Amp>
int gate_plain(qsim *s, const GateRec &g) {
    Amp *psi = (Amp *)s->state;
    const uint64_t tbit = 1ull << g.targets[0];
    switch (g.kind) {
    case GK_PHASE: {
        const uint64_t mask = g.tmask | g.cmask;
        const InsertSpec ins = make_spec(mask);
        const uint64_t ngroups = 1ull << (s->n - ins.m);
        k_phase<Amp><<<blocks_for(ngroups, 256 * kPhaseGroups), 256, 0, s->stream>>>(psi, ngroups, ins, mask, amp<Amp>(g.m[3]));
        break;
    }
    case GK_DIAG1: {
        const InsertSpec ins = make_spec(g.tmask | g.cmask);
        const uint64_t ngroups = 1ull << (s->n - ins.m);
        k_diag1<Amp><<<blocks_for(ngroups, 256 * kGroups), 256, 0, s->stream>>>(psi, ngroups, ins, g.cmask, tbit,
                                                                        amp<Amp>(g.m[0]), amp<Amp>(g.m[3]));
        break;
    }
    case GK_X: {
        const InsertSpec ins = make_spec(g.tmask | g.cmask);
        const uint64_t ngroups = 1ull << (s->n - ins.m);
        k_x<Amp><<<blocks_for(ngroups, 256 * kGroups), 256, 0, s->stream>>>(psi, ngroups, ins, g.cmask, tbit);
        break;
    }
    default: {
        switch (g.t) {
        case 1: {
            Mat1<Amp> M;
            for (int i = 0; i < 4; ++i) M.m[i] = amp<Amp>(g.m[i]);
            const InsertSpec ins = make_spec(g.tmask | g.cmask);
            const uint64_t ngroups = 1ull << (s->n - ins.m);
            k_dense1<Amp><<<blocks_for(ngroups, 256 * kGroups), 256, 0, s->stream>>>(psi, ngroups, ins, g.cmask, tbit, M);
            break;
        }
        case 2: return dense_k<Amp, 2>(s, g.targets, g.cmask, g.m.data());
        case 3: return dense_k<Amp, 3>(s, g.targets, g.cmask, g.m.data());
        case 4: return dense_k<Amp, 4>(s, g.targets, g.cmask, g.m.data());
        case 5: return dense_k<Amp, 5>(s, g.targets, g.cmask, g.m.data());
        default: return set_err(s, QSIM_EINVAL, "gate with more than 5 targets");
        }
    }
    }
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "gate launch");
}

template <typename Amp>
int block_dense(qsim *s, const int *q, int k, const cd *m) {
    if (k == 1) {
        GateRec g;
        g.t = 1;
        g.targets[0] = q[0];
        g.tmask = 1ull << q[0];
        g.m.assign(m, m + 4);
        g.kind = GK_DENSE;
        return launch_gate_plain(s, g);  // applies the double-float choice
    }
    switch (k) {
    case 2: return dense_k<Amp, 2>(s, q, 0, m);
    case 3: return dense_k<Amp, 3>(s, q, 0, m);
    case 4: return dense_k<Amp, 4>(s, q, 0, m);
    case 5: return dense_k<Amp, 5>(s, q, 0, m);
    }
    return set_err(s, QSIM_EINVAL, "block width outside 1..5");
}

template <typename Amp>
__global__ void k_set_basis(Amp *__restrict__ psi, uint64_t N, uint64_t basis) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (; i < N; i += stride) {
        Amp z;
        z.x = (i == basis) ? 1 : 0;
        z.y = 0;
        psi[i] = z;
    }
}

}  // namespace

int launch_gate_plain(qsim *s, const GateRec &g) {
    if (s->prec == QSIM_C128 && s->c128_df && gate_df(s, g)) {
        s->stats.launches++;
        return cuda_err(s, cudaGetLastError(), "double-float gate launch");
    }
    return s->prec == QSIM_C128 ? gate_plain<double2>(s, g) : gate_plain<float2>(s, g);
}

int launch_block_dense(qsim *s, const int *qubits, int k, const cd *m) {
    return s->prec == QSIM_C128 ? block_dense<double2>(s, qubits, k, m) : block_dense<float2>(s, qubits, k, m);
}

int launch_set_basis(qsim *s, uint64_t basis) {
    const uint64_t N = 1ull << s->n;
    const unsigned grid = (unsigned)std::min<uint64_t>(blocks_for(N, 256), (uint64_t)s->sms * 16);
    if (s->prec == QSIM_C128)
        k_set_basis<double2><<<grid, 256, 0, s->stream>>>((double2 *)s->state, N, basis);
    else
        k_set_basis<float2><<<grid, 256, 0, s->stream>>>((float2 *)s->state, N, basis);
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "set basis launch");
}

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
// qubits outside the register and the controls.  When the register holds a
// lower qubit than any run qubit, the accesses are coalesced over the
// register value and a tile holds 2^11 amplitudes (or all of the
// register's 2^m), small enough for eight CTAs per SM; otherwise it holds
// 2^13 and a run is at least 32 bytes (one DRAM sector) where such qubits
// exist.  f acts on every run alike, so a tile maps onto
// itself: the CTA loads it into shared memory (16 loads per thread in flight
// for complex64, 8 for complex128), the index holding the lowest address bit
// varying fastest so that the loads are coalesced whether the register holds
// the low qubits or the high ones; it synchronises, and writes each position
// from its source, out(v, r) = in(f^-1(v), r), so the stores are coalesced
// too.  The register-value offsets (two 64-entry tables for bits 0..5 and
// 6..11 of the value), the run offsets and f^-1 come from a device record
// and are copied to shared memory once per CTA.  m <= 12.
//
// Where the register and the controls lie above the 9 lowest qubits (8 for
// complex128: 4 KB of contiguous amplitudes), the permutation
// instead follows the cycles of f: for a cycle e_0 -> e_1 -> ... -> e_{L-1}
// -> e_0 and a slice of 4 KB at the same place in every register value's
// block, the data rotate one step along the cycle in place,
//   new[e_{i+1}] = old[e_i],
// walked from e_{L-1} down to e_0 with the loads of the next eight elements
// in flight (a load of e_j always precedes the store to e_j).  Every access
// of a CTA is 4 KB contiguous, fixed points of f are not touched, and the
// work is (cycle, slice) tasks, longest cycles first.  Above the lowest 16 KB
// the same walk runs through the bulk-copy engine (k_permute_cycles_bulk).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

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

// six CTAs per SM for complex64 (40 registers, no spills), three for complex128
template <typename Amp>
__global__ void __launch_bounds__(kPermThreads, sizeof(Amp) == 8 ? 6 : 3) k_permute(Amp *__restrict__ psi, uint64_t ntiles, const InsertSpec ins,
                                                          uint64_t cmask, int m, int c, int v_fast,
                                                          const uint64_t *__restrict__ goff,
                                                          const uint64_t *__restrict__ groff,
                                                          const uint32_t *__restrict__ gfinv) {
    // shared memory: the tile, then the tables (register-value offsets as
    // two 64-entry halves, run offsets, f^-1), copied once per CTA
    extern __shared__ unsigned char sm_raw[];
    Amp *buf = (Amp *)sm_raw;
    const unsigned T = 1u << (m + c), D = 1u << m, R = 1u << c;
    uint64_t *olo = (uint64_t *)(sm_raw + sizeof(Amp) * T);
    uint64_t *ohi = olo + 64;
    uint64_t *roff = ohi + 64;
    uint32_t *finv = (uint32_t *)(roff + R);
    for (unsigned i = threadIdx.x; i < 128; i += kPermThreads) olo[i] = goff[i];  // olo and ohi
    for (unsigned i = threadIdx.x; i < D; i += kPermThreads) finv[i] = gfinv[i];
    for (unsigned i = threadIdx.x; i < R; i += kPermThreads) roff[i] = groff[i];
    __syncthreads();
    auto off = [&](unsigned v) { return olo[v & 63u] | ohi[v >> 6]; };
    constexpr int kL = 8;  // loads in flight per thread per round
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
                    a[u] = psi[base + off(v) + roff[r]];
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
            psi[base + off(v) + roff[r]] = buf[v_fast ? ((r << m) | fv) : ((fv << c) | r)];
        }
        __syncthreads();
    }
}

constexpr int kCycThreads = 256;
constexpr int kCycDepth = 8;  // loads in flight per thread along a cycle

// coff: the cycles' elements as register offsets in 16-byte units, cycle
// by cycle, f(e_i) = e_{i+1}; cstart[j]: first element of cycle j (ncyc + 1
// entries); a task is (cycle, slice) with the slice fastest.  The current
// cycle's offsets are copied to shared memory (dynamic, 8 bytes times the
// longest cycle), so the address of each step is one shared-memory read.
__global__ void __launch_bounds__(kCycThreads) k_permute_cycles(float4 *__restrict__ psi16, const InsertSpec ins,
                                                                uint64_t cmask16, const uint64_t *__restrict__ coff,
                                                                const uint32_t *__restrict__ cstart, uint32_t ncyc,
                                                                uint64_t nslices, int amp_shift) {
    extern __shared__ uint64_t s_e[];
    const uint64_t ntasks = (uint64_t)ncyc * nslices;
    uint32_t loaded = 0xffffffffu;  // the cycle whose offsets are in s_e
    for (uint64_t task = blockIdx.x; task < ntasks; task += gridDim.x) {
        const uint32_t cyc = (uint32_t)(task / nslices);
        const uint64_t sl = task - (uint64_t)cyc * nslices;
        const uint32_t b0 = cstart[cyc];
        const int L = (int)(cstart[cyc + 1] - b0);
        if (cyc != loaded) {  // uniform over the CTA
            __syncthreads();
            for (int i = threadIdx.x; i < L; i += kCycThreads) s_e[i] = coff[b0 + i];
            __syncthreads();
            loaded = cyc;
        }
        const uint64_t *e = s_e;
        // this thread's 16 bytes of the slice at register value 0
        float4 *p = psi16 + (((insert_zeros(sl << (8 + amp_shift), ins) >> amp_shift) | cmask16) + threadIdx.x);
        const float4 first = p[e[L - 1]];
        float4 r[kCycDepth];  // r[j] holds old[e_{L-2-j}], then the element kCycDepth further down
#pragma unroll
        for (int j = 0; j < kCycDepth; ++j)
            if (L - 2 - j >= 0) r[j] = p[e[L - 2 - j]];
        int i = L - 1;  // the element written next (from old[e_{i-1}])
        while (i >= 1) {
#pragma unroll
            for (int j = 0; j < kCycDepth; ++j) {
                if (i >= 1) {
                    const float4 v = r[j];
                    if (i - 1 - kCycDepth >= 0) r[j] = p[e[i - 1 - kCycDepth]];
                    p[e[i]] = v;
                    --i;
                }
            }
        }
        p[e[0]] = first;
    }
}

// Cycle walk through the bulk-copy engine, for registers above the lowest
// 16 KB of amplitudes: one thread per CTA moves 16 KB slices with
// cp.async.bulk, global -> shared stage (completing on the stage's
// mbarrier) -> global, kBulkStages loads ahead, so the bytes in flight are
// bounded by shared memory rather than registers.  For a cycle x_j =
// e_{L-1-j}: x_0 goes to its own buffer; at step j >= 1 the thread waits for
// x_j's stage, stores it to x_{j-1} (whose load completed at step j - 1),
// and refills the stage the store of step j - 1 has finished reading with
// x_{j+S-1}; last, x_0's data goes to x_{L-1} = e_0.  Each element is read
// before it is written and every wait is bounded (time-out: error flag,
// bounded waits for the copies in flight, return).
constexpr int kBulkStages = 4;
constexpr uint32_t kBulkSlice = 16384;  // bytes per slice (one bulk copy)

__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(qsim_tc::smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// coff32: the cycles' register offsets in slice units, cycle by cycle;
// dynamic shared memory: (kBulkStages + 1) slices, then the current cycle's
// offsets (uint32, the longest cycle).
__global__ void __launch_bounds__(32) k_permute_cycles_bulk(unsigned char *__restrict__ psi, const InsertSpec ins,
                                                           uint64_t cmask, int amp_bytes, int slice_bits,
                                                           const uint32_t *__restrict__ coff32,
                                                           const uint32_t *__restrict__ cstart, uint32_t ncyc,
                                                           uint64_t nslices, unsigned int *err) {
    extern __shared__ __align__(128) unsigned char sm_bulk[];
    __shared__ __align__(8) uint64_t bar[kBulkStages + 1];  // [kBulkStages]: x_0's buffer
    unsigned char *stage = sm_bulk;                           // kBulkStages + 1 slices
    uint32_t *s_off = (uint32_t *)(sm_bulk + (size_t)(kBulkStages + 1) * kBulkSlice);
    if (threadIdx.x == 0) {
        for (int i = 0; i <= kBulkStages; ++i) qsim_tc::mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    uint32_t parity = 0;  // bit i: the phase barrier i waits for next (thread 0)
    const uint64_t ntasks = (uint64_t)ncyc * nslices;
    uint32_t loaded = 0xffffffffu;
    for (uint64_t task = blockIdx.x; task < ntasks; task += gridDim.x) {
        const uint32_t cyc = (uint32_t)(task / nslices);
        const uint64_t sl = task - (uint64_t)cyc * nslices;
        const uint32_t b0 = cstart[cyc];
        const int L = (int)(cstart[cyc + 1] - b0);
        if (cyc != loaded) {
            for (int i = threadIdx.x; i < L; i += 32) s_off[i] = coff32[b0 + i];
            loaded = cyc;
        }
        __syncwarp();
        bool ok = true;
        if (threadIdx.x == 0) {
            unsigned char *base = psi + (insert_zeros(sl << slice_bits, ins) | cmask) * (uint64_t)amp_bytes;
            auto addr = [&](int j) { return base + (uint64_t)s_off[L - 1 - j] * kBulkSlice; };  // x_j
            auto load = [&](int b, int j) {
                qsim_tc::mbar_expect_tx(&bar[b], kBulkSlice);
                qsim_tc::bulk_copy(stage + (size_t)b * kBulkSlice, addr(j), kBulkSlice, &bar[b]);
            };
            auto wait = [&](int b) {
                const bool r = qsim_tc::mbar_wait(&bar[b], (parity >> b) & 1u);
                parity ^= 1u << b;
                return r;
            };
            uint32_t pending = 1u << kBulkStages;  // barriers with a load in flight
            load(kBulkStages, 0);
            for (int j = 1; j < kBulkStages && j < L; ++j) {
                load(j % kBulkStages, j);
                pending |= 1u << (j % kBulkStages);
            }
            ok = wait(kBulkStages);
            pending &= ~(1u << kBulkStages);
            for (int j = 1; ok && j < L; ++j) {
                const int b = j % kBulkStages;
                ok = wait(b);
                pending &= ~(1u << b);
                if (!ok) break;
                qsim_tc::fence_proxy_async_smem();
                bulk_store(addr(j - 1), stage + (size_t)b * kBulkSlice, kBulkSlice);
                const int nx = j + kBulkStages - 1;
                if (nx < L) {
                    bulk_wait_read_1();  // the previous store has read its stage
                    load(nx % kBulkStages, nx);
                    pending |= 1u << (nx % kBulkStages);
                }
            }
            if (ok) bulk_store(addr(L - 1), stage + (size_t)kBulkStages * kBulkSlice, kBulkSlice);
            bulk_wait_all();
            if (!ok) {
                atomicOr(err, 1u);
                for (int b = 0; b <= kBulkStages; ++b)
                    if ((pending >> b) & 1u) wait(b);  // the loads still in flight, bounded
            }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) return;
    }
}

// The cycle walk when the register and the controls leave the lowest 4 KB
// of amplitudes contiguous and there are enough tasks to fill the GPU;
// returns QSIM_ENOTSUP otherwise (the tiled kernel then runs).
template <typename Amp>
int permute_cycles(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask,
                   bool *bulk) {
    *bulk = false;
    const int amp_shift = sizeof(Amp) == 8 ? 1 : 0;  // amplitudes per 16 bytes: 2 or 1
    const int slice_bits = 8 + amp_shift;  // 4 KB slices: 512 c64 or 256 c128 amplitudes
    const int bulk_bits = slice_bits + 2;  // 16 KB slices for the bulk-copy walk
    const uint64_t fixed = qmask | cmask;
    if ((fixed & ((1ull << slice_bits) - 1ull)) != 0) return QSIM_ENOTSUP;
    const int D = 1 << m;
    // the cycles of f, longest first
    std::vector<std::vector<uint32_t>> cycles;
    std::vector<char> seen(D, 0);
    size_t total = 0;
    for (int v = 0; v < D; ++v) {
        if (seen[v] || (int)perm[v] == v) continue;
        std::vector<uint32_t> cy;
        for (uint32_t x = (uint32_t)v; !seen[x]; x = (uint32_t)perm[x]) {
            seen[x] = 1;
            cy.push_back(x);
        }
        total += cy.size();
        cycles.push_back(std::move(cy));
    }
    if (cycles.empty()) return QSIM_OK;  // f is the identity
    const int nfree = s->n - m - __builtin_popcountll(cmask);
    const uint64_t nslices = 1ull << (nfree - slice_bits);
    if ((uint64_t)cycles.size() * nslices < (uint64_t)s->sms) return QSIM_ENOTSUP;
    // the bulk-copy walk: 16 KB slices, at least two tasks per SM
    const bool use_bulk = (fixed & ((1ull << bulk_bits) - 1ull)) == 0 && nfree >= bulk_bits &&
                          (uint64_t)cycles.size() * (1ull << (nfree - bulk_bits)) >= 2ull * (uint64_t)s->sms;
    std::stable_sort(cycles.begin(), cycles.end(),
                     [](const std::vector<uint32_t> &a, const std::vector<uint32_t> &b) { return a.size() > b.size(); });
    const size_t ncyc = cycles.size();
    InsertSpec ins{};
    ins.m = 0;
    for (int b = 0; b < 64; ++b)
        if ((fixed >> b) & 1ull) ins.pos[ins.m++] = b;
    if (use_bulk) {
        // record: offsets in 16 KB slice units (uint32), then cycle starts
        const size_t bslice_amps = (size_t)kBulkSlice / sizeof(Amp);
        std::vector<uint32_t> rb(total + ncyc + 1);
        size_t k = 0;
        for (size_t j = 0; j < ncyc; ++j) {
            rb[total + j] = (uint32_t)k;
            for (uint32_t v : cycles[j]) {
                uint64_t a = 0;
                for (int b = 0; b < m; ++b)
                    if ((v >> b) & 1u) a |= 1ull << qubits[b];
                rb[k++] = (uint32_t)(a / bslice_amps);
            }
        }
        rb[total + ncyc] = (uint32_t)k;
        unsigned char *dev = nullptr;
        int rc = stage_operand(s, rb.data(), rb.size() * sizeof(uint32_t), &dev);
        if (rc) return rc;
        const uint64_t bslices = 1ull << (nfree - bulk_bits);
        const uint64_t ntasks = (uint64_t)ncyc * bslices;
        const size_t smem = (size_t)(kBulkStages + 1) * kBulkSlice + sizeof(uint32_t) * cycles[0].size();
        static bool attr[64] = {false};
        if (s->device >= 0 && s->device < 64 && !attr[s->device]) {
            cudaError_t e = cudaFuncSetAttribute(k_permute_cycles_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)((kBulkStages + 1) * kBulkSlice + sizeof(uint32_t) * 4096));
            if (e != cudaSuccess) return cuda_err(s, e, "permutation kernel attribute");
            attr[s->device] = true;
        }
        // two CTAs (one pipeline each) per SM
        const uint64_t grid = ntasks < (uint64_t)s->sms * 2 ? ntasks : (uint64_t)s->sms * 2;
        k_permute_cycles_bulk<<<(unsigned)grid, 32, smem, s->stream>>>(
            (unsigned char *)s->state, ins, cmask, (int)sizeof(Amp), bulk_bits, (const uint32_t *)dev,
            (const uint32_t *)dev + total, (uint32_t)ncyc, bslices, (unsigned int *)((char *)s->ws + kWsErr));
        s->stats.launches++;
        *bulk = true;
        return cuda_err(s, cudaGetLastError(), "permutation launch");
    }
    std::vector<unsigned char> rec(sizeof(uint64_t) * total + sizeof(uint32_t) * (ncyc + 1));
    uint64_t *coff = (uint64_t *)rec.data();
    uint32_t *cstart = (uint32_t *)(rec.data() + sizeof(uint64_t) * total);
    size_t k = 0;
    for (size_t j = 0; j < ncyc; ++j) {
        cstart[j] = (uint32_t)k;
        for (uint32_t v : cycles[j]) {
            uint64_t a = 0;
            for (int b = 0; b < m; ++b)
                if ((v >> b) & 1u) a |= 1ull << qubits[b];
            coff[k++] = a >> amp_shift;
        }
    }
    cstart[ncyc] = (uint32_t)k;
    unsigned char *dev = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev);
    if (rc) return rc;
    const uint64_t ntasks = (uint64_t)ncyc * nslices;
    // 64 registers a thread: four CTAs of 256 threads resident per SM
    const uint64_t grid = ntasks < (uint64_t)s->sms * 4 ? ntasks : (uint64_t)s->sms * 4;
    const size_t smem = sizeof(uint64_t) * cycles[0].size();  // the longest cycle (<= 2^12 entries)
    k_permute_cycles<<<(unsigned)grid, kCycThreads, smem, s->stream>>>(
        (float4 *)s->state, ins, cmask >> amp_shift, (const uint64_t *)dev,
        (const uint32_t *)(dev + sizeof(uint64_t) * total), (uint32_t)ncyc, nslices, amp_shift);
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "permutation launch");
}

template <typename Amp>
int permute(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask) {
    const int D = 1 << m;
    const int n = s->n;
    // run qubits: the lowest outside the register and the controls
    const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    const uint64_t free = all & ~(qmask | cmask);
    // the index holding the lowest address bit varies fastest: the register
    // value when the register holds a lower qubit than any run qubit; then
    // the loads and stores are coalesced over v and tiles of 2^11 amplitudes
    // suffice (small tiles: many CTAs per SM); else runs of at least one
    // 32-byte sector in tiles of 2^13
    const bool v_fast = free == 0 || (qmask & (0ull - qmask)) < (free & (0ull - free));
    const int cmin = v_fast ? 0 : (sizeof(Amp) == 8 ? 2 : 1);
    const int tile_bits = v_fast ? 11 : 13;
    int c = tile_bits - m < cmin ? cmin : tile_bits - m;
    while (c > 0 && ((size_t)sizeof(Amp) << (m + c)) > kPermSmemMax) --c;
    if (c > __builtin_popcountll(free)) c = __builtin_popcountll(free);
    int rbit[64], nr = 0;
    for (int b = 0; b < n && nr < c; ++b)
        if ((free >> b) & 1ull) rbit[nr++] = b;
    uint64_t rmask = 0;
    for (int j = 0; j < c; ++j) rmask |= 1ull << rbit[j];
    const int R = 1 << c;
    // record: olo[64], ohi[64] (register-value offsets of bits 0..5 and
    // 6..11 of v), roff[R], finv[D]
    std::vector<unsigned char> rec(sizeof(uint64_t) * (128 + R) + sizeof(uint32_t) * D);
    uint64_t *olo = (uint64_t *)rec.data();
    uint64_t *ohi = olo + 64;
    uint64_t *roff = ohi + 64;
    uint32_t *finv = (uint32_t *)(rec.data() + sizeof(uint64_t) * (128 + R));
    auto reg_off = [&](int v) {
        uint64_t a = 0;
        for (int j = 0; j < m; ++j)
            if ((v >> j) & 1) a |= 1ull << qubits[j];
        return a;
    };
    for (int v = 0; v < 64; ++v) {
        olo[v] = reg_off(v & (D - 1));
        ohi[v] = (v << 6) < D ? reg_off(v << 6) : 0;
    }
    for (int v = 0; v < D; ++v) finv[perm[v]] = (uint32_t)v;
    for (int r = 0; r < R; ++r) {
        uint64_t a = 0;
        for (int j = 0; j < c; ++j)
            if ((r >> j) & 1) a |= 1ull << rbit[j];
        roff[r] = a;
    }
    unsigned char *dev = nullptr;
    int rc = stage_operand(s, rec.data(), rec.size(), &dev);
    if (rc) return rc;
    InsertSpec ins{};
    ins.m = 0;
    const uint64_t fixed = qmask | cmask | rmask;
    for (int b = 0; b < 64; ++b)
        if ((fixed >> b) & 1ull) ins.pos[ins.m++] = b;
    const uint64_t ntiles = 1ull << (n - ins.m);
    const size_t smem = (sizeof(Amp) << (m + c)) + sizeof(uint64_t) * (128 + R) + sizeof(uint32_t) * D;
    static bool attr[2][64] = {{false}};
    const int which = sizeof(Amp) == 8 ? 0 : 1;
    if (s->device >= 0 && s->device < 64 && !attr[which][s->device]) {
        cudaError_t e = cudaFuncSetAttribute(k_permute<Amp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kPermSmemMax + sizeof(uint64_t) * (128 + 4096) + 4 * 4096));
        if (e != cudaSuccess) return cuda_err(s, e, "permutation kernel attribute");
        attr[which][s->device] = true;
    }
    const uint64_t grid = ntiles < (uint64_t)s->sms * 8 ? ntiles : (uint64_t)s->sms * 8;
    k_permute<Amp><<<(unsigned)grid, kPermThreads, smem, s->stream>>>(
        (Amp *)s->state, ntiles, ins, cmask, m, c, v_fast ? 1 : 0, (const uint64_t *)dev,
        (const uint64_t *)dev + 128, (const uint32_t *)(dev + sizeof(uint64_t) * (128 + R)));
    s->stats.launches++;
    return cuda_err(s, cudaGetLastError(), "permutation launch");
}

}  // namespace

int launch_permutation(qsim *s, const uint64_t *perm, const int *qubits, int m, uint64_t qmask, uint64_t cmask,
                       int *kind) {
    const bool c128 = s->prec == QSIM_C128;
    bool bulk = false;
    int rc = c128 ? permute_cycles<double2>(s, perm, qubits, m, qmask, cmask, &bulk)
                  : permute_cycles<float2>(s, perm, qubits, m, qmask, cmask, &bulk);
    *kind = rc == QSIM_ENOTSUP ? 0 : bulk ? 2 : 1;
    if (rc != QSIM_ENOTSUP) return rc;
    return c128 ? permute<double2>(s, perm, qubits, m, qmask, cmask) : permute<float2>(s, perm, qubits, m, qmask, cmask);
}

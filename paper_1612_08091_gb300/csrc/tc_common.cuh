// tc_common.cuh -- inline-PTX helpers shared by the tensor-core block
// kernels (fused_kernel.cu: 5-qubit blocks, tmem_block_kernel.cu: 5- and 6-qubit
// blocks) and the batched variational kernel (vqe_kernel.cu: bulk copies):
// mbarriers with bounded waits, bulk copies, tcgen05 fences, shared-memory
// matrix descriptors, MMA commit, tensor-memory loads and stores, and the
// bf16 hi/lo split of an amplitude.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

namespace qsim_tc {

// Upper bound on the polls of one mbarrier wait.  Every wait in the block
// kernels gives up after it, raises an error flag and lets the kernel free
// its tensor memory and return.  A poll of a barrier that never completes
// took 3.9 us on GB300 (qsim_selftest_wait_timeout), so 2^18 polls give up
// after about one second; the copies and tensor-core commits waited for
// take microseconds.
constexpr uint32_t kWaitLimit = 1u << 18;

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

// Bounded wait (at most `limit` polls); returns false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Arrive on `bar` (count 1) and add `bytes` to the transaction count its
// current phase waits for.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk copy global -> shared of `bytes` (16-byte aligned addresses, a
// multiple of 16 bytes), completing its bytes on `bar`.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// One bulk copy global -> shared completing on `bar` (which expects `bytes`).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    mbar_expect_tx(bar, bytes);
    bulk_copy(dst, src, bytes, bar);
}

// Order this thread's earlier generic-proxy accesses (to global memory, or
// to this CTA's shared memory) before its later async-proxy (bulk copy)
// accesses.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

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

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major.
constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes; the wait is in
// the same asm statement, so the registers are complete when it returns
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (thread i of
// the warp writes lane i); tcgen05_wait_st() makes them complete
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *w) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]),
        "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
        : "memory");
}
// 16 lanes x 16 consecutive 32-bit columns (shape 16x256b, two
// repetitions of 8 columns).  Thread t of the warp holds, for repetition
// rep, columns 8 rep + 2 (t & 3) and + 1 of lane (t >> 2) in w[4 rep],
// w[4 rep + 1] and the same columns of lane (t >> 2) + 8 in w[4 rep + 2],
// w[4 rep + 3]: the four threads of a quad share two lanes.
__device__ __forceinline__ void tmem_st16x256b_x2(uint32_t taddr, const uint32_t *w) {
    asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// The same fragment with four repetitions (32 columns), read and waited for
__device__ __forceinline__ void tmem_ld16x256b_x4(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tcgen05_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_half, float hi_half) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo_half, hi_half);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// Split (re, im) into bf16 hi = round-to-nearest and lo = round-to-nearest
// bf16 of the exact remainder x - hi (hi + lo carries x to 2^-16 relative).
// Each word packs re in its low half and im in its high half, i.e. the two
// consecutive K elements 2r, 2r+1 of an operand row.  A truncated hi costs
// the same instructions but biases the dropped lo x lo product and doubles
// the norm drift, so hi is rounded.
__device__ __forceinline__ void split_pair(float re, float im, uint32_t &hw, uint32_t &lw) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    memcpy(&hw, &h, 4);
    const float rr = re - __uint_as_float(hw << 16);
    const float ri = im - __uint_as_float(hw & 0xFFFF0000u);
    lw = pack_bf16x2(rr, ri);
}

// Host side: round-to-nearest-even bf16 of a float (finite inputs), and the
// bf16 value back as a double; the operand records split the gate matrix
// with these in FP64 (R1 = bf16(R), R2 = bf16(R - R1), ...).
inline uint16_t f32_to_bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t round = 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)((u + round) >> 16);
}
inline double bf16_bits_to_double(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

}  // namespace qsim_tc

// common.cuh -- device-side helpers shared by the libqsim kernels.
//
// Amplitudes are interleaved complex numbers: double2 for complex128 and
// float2 for complex64.  Qubit q is bit q of the amplitude index.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsim_dev {

constexpr int kMaxQubits = 36;     // largest register the library accepts

// Sorted list of bit positions to insert (as zeros) into a group counter so
// that it enumerates the basis indices with those bits cleared.
struct InsertSpec {
    int m;            // number of positions
    int pos[kMaxQubits];
};

// Spread the bits of g around the sorted zero positions p[0] < p[1] < ...:
// the result has a 0 at each p[j] and the bits of g, in order, elsewhere.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t g, const InsertSpec &s) {
    for (int j = 0; j < s.m; ++j) {
        const int p = s.pos[j];
        const uint64_t low = g & ((1ull << p) - 1ull);
        g = ((g >> p) << (p + 1)) | low;
    }
    return g;
}

// complex helpers -----------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// acc + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

template <typename A> struct AmpTraits;
template <> struct AmpTraits<double2> { typedef double real; };
template <> struct AmpTraits<float2> { typedef float real; };

// |a|^2 in the amplitude's own precision
__device__ __forceinline__ double norm2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float norm2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace qsim_dev

// df128.cuh -- complex128 gate arithmetic in pairs of FP32 ("double-float").
//
// GB300 executes FP64 fused multiply-adds at about 1/58 of the FP32 rate
// (measured 1.2 TFLOP/s against 70 TFLOP/s), so a one-qubit gate on complex128
// amplitudes with FP64 arithmetic (8 FMAs per amplitude) runs at a third of
// the HBM bandwidth.  In this mode each double is split, with integer bit
// operations only, into hi + lo floats (24 + 23 significant bits, relative
// truncation error <= 2^-46); products are formed exactly with FMA
// (p = uh*xh, e = fma(uh, xh, -p)) plus the two cross terms; four products
// are summed with error-free two-sums; the (hi, lo) result is widened to
// double exactly with integer operations and added with one FP64 add, which
// also rounds it to double.  The relative error per result is about 2^-45
// (1e-14) instead of FP64's 2^-53, for two FP64 adds per amplitude.
// Magnitudes below 2^-126 (hi) or 2^-80 (lo) are flushed to zero, an
// absolute error below 1e-24 for state amplitudes and gate entries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsim_df {

struct F2 {  // value = hi + lo
    float hi, lo;
};

// x -> hi + lo with integer operations (no FP64 instruction)
__device__ __forceinline__ F2 split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const int e = (int)((h32 >> 20) & 0x7FFu);
    const unsigned sgn = h32 & 0x80000000u;
    F2 r;
    // hi: the top 24 significant bits (truncated)
    const unsigned hb = sgn | ((unsigned)(e - 896) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
    r.hi = (e >= 897 && e <= 1150) ? __uint_as_float(hb) : 0.f;
    // lo: the next 23 bits, (l32 & (2^29 - 1)) >> 6, times 2^(e - 1069)
    const unsigned m = (l32 & 0x1FFFFFFFu) >> 6;
    const float fm = __uint_as_float(0x4B000000u | m) - 8388608.0f;  // exactly m
    const int pe = e - 942;                                            // biased exponent of 2^(e-1069)
    const float p2 = __uint_as_float((unsigned)(pe > 0 ? pe : 0) << 23);
    r.lo = (pe >= 1 && e >= 897 && e <= 1150) ? __uint_as_float(__float_as_uint(fm * p2) | sgn) : 0.f;
    return r;
}

// exact widening of a normal float (denormals flushed) to double bits
__device__ __forceinline__ double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e8 = (b >> 23) & 0xFFu;
    const unsigned h32 = (b & 0x80000000u) | ((e8 + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    const unsigned l32 = b << 29;
    const unsigned long long bits = ((unsigned long long)h32 << 32) | l32;
    return e8 ? __longlong_as_double((long long)bits) : 0.0;
}

// hi + lo rounded to double (one FP64 add)
__device__ __forceinline__ double to_double(F2 v) { return widen(v.hi) + widen(v.lo); }

// u * x as an unnormalised pair (p exact product of the highs, q the rest)
__device__ __forceinline__ F2 mul(F2 u, F2 x) {
    F2 r;
    r.hi = u.hi * x.hi;
    const float e = fmaf(u.hi, x.hi, -r.hi);
    r.lo = fmaf(u.hi, x.lo, fmaf(u.lo, x.hi, e));
    return r;
}

// a + b with the rounding error of the highs carried in lo (two-sum)
__device__ __forceinline__ F2 add(F2 a, F2 b) {
    F2 r;
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    r.hi = s;
    r.lo = a.lo + b.lo + err;
    return r;
}

__device__ __forceinline__ F2 neg(F2 a) {
    a.hi = -a.hi;
    a.lo = -a.lo;
    return a;
}

// complex number of double-float parts
struct C2 {
    F2 re, im;
};

__device__ __forceinline__ C2 split(double2 z) { return C2{split(z.x), split(z.y)}; }
__device__ __forceinline__ double2 to_double(const C2 &z) { return make_double2(to_double(z.re), to_double(z.im)); }

// u0 * x0 + u1 * x1 (complex)
__device__ __forceinline__ C2 cdot2(const C2 &u0, const C2 &x0, const C2 &u1, const C2 &x1) {
    C2 r;
    r.re = add(add(mul(u0.re, x0.re), neg(mul(u0.im, x0.im))), add(mul(u1.re, x1.re), neg(mul(u1.im, x1.im))));
    r.im = add(add(mul(u0.re, x0.im), mul(u0.im, x0.re)), add(mul(u1.re, x1.im), mul(u1.im, x1.re)));
    return r;
}

// a + b (complex)
__device__ __forceinline__ C2 cadd(const C2 &a, const C2 &b) { return C2{add(a.re, b.re), add(a.im, b.im)}; }

// u * x (complex)
__device__ __forceinline__ C2 cmul(const C2 &u, const C2 &x) {
    C2 r;
    r.re = add(mul(u.re, x.re), neg(mul(u.im, x.im)));
    r.im = add(mul(u.re, x.im), mul(u.im, x.re));
    return r;
}

}  // namespace qsim_df

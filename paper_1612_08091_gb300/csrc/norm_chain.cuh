// norm_chain.cuh -- the norm control shared by the passes that compute in
// reduced precision (the tensor-core block passes of tmem_block_kernel.cu
// and the product passes of product_kernel.cu).
//
// Every such pass writes per-CTA FP64 sums of |x|^2 over its inputs (a)
// and of |y|^2 over its raw outputs (b), and CTA 0 records the scale s it
// applied and the norm target T.  The next pass knows the norm the previous
// one left, s^2 b, and its shrink ratio b / a; assuming the same ratio, it
// scales its outputs by
//     s' = sqrt(T / (s^2 b * b / a)),
// which brings the norm back to T after every pass.  T is 1 after a reset
// or a measurement and the input norm of the first pass otherwise; the host
// starts a new chain (no previous record, scale 1) where the norm changes.
// The sums of two consecutive passes live in two slots of the workspace.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace qsim_chain {

struct ChainArgs {
    double *norm_out;         // this pass: per-CTA input sums at [0, grid), output sums at [kMaxTcGrid, ...)
    double *rec_out;          // {scale applied, target}, written by CTA 0
    const double *norm_prev;  // the previous pass's sums (prev_grid CTAs); null starts a chain
    const double *rec_prev;   // its record; null starts a chain
    double target;            // a new chain's target (<= 0: this pass's own input norm)
    int prev_grid;
};

// The output scale of this pass (every CTA's thread 0 computes the same
// value: fixed summation order); CTA 0 also writes the record.
__device__ inline float chain_scale(const ChainArgs &c) {
    float sc = 1.0f;
    double T = c.target;
    if (c.norm_prev) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < c.prev_grid; ++i) {
            a += c.norm_prev[i];
            b += c.norm_prev[kMaxTcGrid + i];
        }
        const double sp = c.rec_prev[0], tp = c.rec_prev[1];
        T = tp > 0.0 ? tp : a;
        if (T > 0.0 && a > 0.0 && b > 0.0 && sp > 0.0 && a < 1e300 && b < 1e300 && T < 1e300) {
            const double s2 = (T / (sp * sp * b)) * (a / b);
            // a correction this large means the chain was not restarted
            // where the norm changed; leave the pass unscaled
            if (s2 > 0.25 && s2 < 4.0) sc = (float)sqrt(s2);
        }
    }
    if (blockIdx.x == 0 && c.rec_out) {
        c.rec_out[0] = (double)sc;
        c.rec_out[1] = T;
    }
    return sc;
}

// This CTA's sums (called by one thread).
__device__ inline void chain_sums(const ChainArgs &c, double in, double out) {
    if (!c.norm_out) return;
    c.norm_out[blockIdx.x] = in;
    c.norm_out[kMaxTcGrid + blockIdx.x] = out;
}

// Host: the chain arguments of the next pass on s.
inline ChainArgs chain_next(const qsim *s) {
    double *slots = (double *)((char *)s->ws + kWsNorm);
    double *recs = slots + 4 * kMaxTcGrid;
    const int slot = (int)(s->tc_passes & 1);
    const bool chain = s->norm_tracking && s->norm_chain;
    ChainArgs c;
    c.norm_out = slots + slot * 2 * kMaxTcGrid;
    c.rec_out = recs + 2 * slot;
    c.norm_prev = chain ? slots + (slot ^ 1) * 2 * kMaxTcGrid : nullptr;
    c.rec_prev = chain ? recs + 2 * (slot ^ 1) : nullptr;
    c.target = s->norm_target;
    c.prev_grid = s->tc_prev_grid;
    return c;
}

// Host: after the pass's launch with `grid` CTAs.
inline void chain_advance(qsim *s, int grid) {
    s->tc_passes++;
    s->tc_prev_grid = grid;
    s->norm_chain = true;
}

}  // namespace qsim_chain

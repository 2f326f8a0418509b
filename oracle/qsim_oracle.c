/*
 * qsim_oracle.c -- plain, unfused FP64 dense state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the GPU
 * library: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path.  It is deliberately slow and literal: every routine is the
 * textbook definition written as a loop over all 2^n basis indices, in
 * complex double, with no blocking, fusion or reordering.
 *
 * What it follows (ProjectQ paper, arXiv:1612.08091):
 *   - gate application to the simulated register, one gate at a time
 *     (Sec. 4.3.2 "Simulation of quantum circuits"; gates act as operators on
 *     the qubits named on the right of '|', Sec. 4);
 *   - controlled gates act only where every control qubit is |1>
 *     (Sec. 4.1.3, the Control meta-instruction);
 *   - measurement in the computational basis with collapse of the register
 *     (Sec. 4 minimal example; Appendix A.1 teleportation, A.3 Shor's
 *     measure-and-reset loop).
 * Conventions the paper leaves open (stated once here, used everywhere):
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - for a gate on targets t[0..k-1], row/column r of its 2^k x 2^k matrix
 *     has bit j of r equal to the value of qubit t[j];
 *   - matrices are row-major complex double;
 *   - single-qubit measurement returns 0 iff u * norm < P(0), where norm is
 *     the squared norm of the register (u is the caller's uniform draw);
 *   - full-register sampling returns the smallest j with
 *     sum_{i<=j} |psi_i|^2 > u * norm.
 *
 * Every routine returns 0 on success or a negative error code (bad qubit
 * index, repeated qubit, zero-probability projection).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

enum { OR_OK = 0, OR_EINVAL = -1, OR_ERANGE = -2, OR_EDUP = -3, OR_EZEROPROB = -4, OR_ENOMEM = -5 };

/* Check that all qubits named are in [0, n) and pairwise distinct, and build
 * their bit mask. */
static int check_qubits(int n, const int *a, int na, const int *b, int nb, uint64_t *mask_a, uint64_t *mask_b)
{
    uint64_t seen = 0, ma = 0, mb = 0;
    for (int j = 0; j < na; ++j) {
        if (a[j] < 0 || a[j] >= n) return OR_ERANGE;
        if (seen & (1ull << a[j])) return OR_EDUP;
        seen |= 1ull << a[j];
        ma |= 1ull << a[j];
    }
    for (int j = 0; j < nb; ++j) {
        if (b[j] < 0 || b[j] >= n) return OR_ERANGE;
        if (seen & (1ull << b[j])) return OR_EDUP;
        seen |= 1ull << b[j];
        mb |= 1ull << b[j];
    }
    *mask_a = ma;
    *mask_b = mb;
    return OR_OK;
}

/* Index of basis state |base> with the target qubits set to the bits of r:
 * bit j of r goes to qubit targets[j]. */
static uint64_t with_targets(uint64_t base, const int *targets, int k, uint64_t r)
{
    uint64_t i = base;
    for (int j = 0; j < k; ++j)
        if ((r >> j) & 1u) i |= 1ull << targets[j];
    return i;
}

/* Apply a k-target gate U (2^k x 2^k, row-major) conditioned on all control
 * qubits being |1>:  for every basis index whose target bits are 0 and whose
 * control bits are 1, gather the 2^k amplitudes it spans, multiply by U,
 * scatter them back.  Indices with a control bit 0 are untouched. */
int or_apply(cplx *psi, int n, const cplx *U, const int *targets, int k, const int *controls, int c)
{
    if (n < 1 || n > 40 || k < 1 || k > 8 || c < 0) return OR_EINVAL;
    uint64_t tmask, cmask;
    int rc = check_qubits(n, targets, k, controls, c, &tmask, &cmask);
    if (rc) return rc;
    const uint64_t N = 1ull << n, D = 1ull << k;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)N; ++i) {
        uint64_t base = (uint64_t)i;
        if ((base & tmask) != 0 || (base & cmask) != cmask) continue;
        cplx in[256], out[256];
        for (uint64_t r = 0; r < D; ++r) in[r] = psi[with_targets(base, targets, k, r)];
        for (uint64_t r = 0; r < D; ++r) {
            cplx s = 0;
            for (uint64_t col = 0; col < D; ++col) s += U[r * D + col] * in[col];
            out[r] = s;
        }
        for (uint64_t r = 0; r < D; ++r) psi[with_targets(base, targets, k, r)] = out[r];
    }
    return OR_OK;
}

/* Squared norm sum_i |psi_i|^2. */
double or_norm2(const cplx *psi, int n)
{
    const uint64_t N = 1ull << n;
    double s = 0.0;
    for (uint64_t i = 0; i < N; ++i) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s;
}

/* Probability mass of the basis states whose listed qubits carry the listed
 * bits: sum over {i : bit qubits[j] of i == bits[j] for all j} of |psi_i|^2. */
int or_prob_bits(const cplx *psi, int n, const int *qubits, int m, const int *bits, double *out)
{
    uint64_t qmask, dummy;
    int rc = check_qubits(n, qubits, m, NULL, 0, &qmask, &dummy);
    if (rc) return rc;
    uint64_t want = 0;
    for (int j = 0; j < m; ++j) {
        if (bits[j] != 0 && bits[j] != 1) return OR_EINVAL;
        if (bits[j]) want |= 1ull << qubits[j];
    }
    const uint64_t N = 1ull << n;
    double s = 0.0;
    for (uint64_t i = 0; i < N; ++i)
        if ((i & qmask) == want) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    *out = s;
    return OR_OK;
}

/* Project onto the subspace where qubits[j] == bits[j] and renormalise by
 * 1/sqrt(p).  A zero-probability projection leaves psi unchanged and returns
 * OR_EZEROPROB.  If p_out is non-NULL it receives p (before renormalising). */
int or_collapse(cplx *psi, int n, const int *qubits, int m, const int *bits, double *p_out)
{
    double p;
    int rc = or_prob_bits(psi, n, qubits, m, bits, &p);
    if (rc) return rc;
    if (p_out) *p_out = p;
    if (!(p > 0.0)) return OR_EZEROPROB;
    uint64_t qmask = 0, want = 0;
    for (int j = 0; j < m; ++j) {
        qmask |= 1ull << qubits[j];
        if (bits[j]) want |= 1ull << qubits[j];
    }
    const double scale = 1.0 / sqrt(p);
    const uint64_t N = 1ull << n;
    for (uint64_t i = 0; i < N; ++i) psi[i] = ((i & qmask) == want) ? psi[i] * scale : 0.0;
    return OR_OK;
}

/* Measure one qubit: outcome 0 iff u * norm < P(qubit = 0), then collapse. */
int or_measure(cplx *psi, int n, int q, double u, int *outcome, double *p_outcome)
{
    if (q < 0 || q >= n) return OR_ERANGE;
    if (!(u >= 0.0 && u < 1.0)) return OR_EINVAL;
    int zero = 0;
    double p0;
    int rc = or_prob_bits(psi, n, &q, 1, &zero, &p0);
    if (rc) return rc;
    const double norm = or_norm2(psi, n);
    int b = (u * norm < p0) ? 0 : 1;
    *outcome = b;
    return or_collapse(psi, n, &q, 1, &b, p_outcome);
}

/* Sample the whole register: with the running sum c_j = sum_{i<=j} |psi_i|^2
 * taken in index order, the outcome is the smallest j with c_j > u * norm.
 * If rounding leaves no such j, the last index of non-zero probability is
 * taken.  The register collapses to |j> with the phase of psi_j kept. */
int or_measure_all(cplx *psi, int n, double u, uint64_t *outcome)
{
    if (!(u >= 0.0 && u < 1.0)) return OR_EINVAL;
    const uint64_t N = 1ull << n;
    const double norm = or_norm2(psi, n);
    if (!(norm > 0.0)) return OR_EZEROPROB;
    const double target = u * norm;
    double c = 0.0;
    uint64_t j = N, last_nonzero = N;
    for (uint64_t i = 0; i < N; ++i) {
        double w = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        if (w > 0.0) last_nonzero = i;
        c += w;
        if (c > target) { j = i; break; }
    }
    if (j == N) j = last_nonzero;
    cplx a = psi[j];
    double mag = cabs(a);
    for (uint64_t i = 0; i < N; ++i) psi[i] = 0.0;
    psi[j] = a / mag;
    *outcome = j;
    return OR_OK;
}

/* Inner product <a|b> = sum_i conj(a_i) b_i. */
void or_inner(const cplx *a, const cplx *b, int n, double *re, double *im)
{
    const uint64_t N = 1ull << n;
    cplx s = 0.0;
    for (uint64_t i = 0; i < N; ++i) s += conj(a[i]) * b[i];
    *re = creal(s);
    *im = cimag(s);
}

/* Set psi to the basis state |x>. */
int or_set_basis(cplx *psi, int n, uint64_t x)
{
    const uint64_t N = 1ull << n;
    if (x >= N) return OR_ERANGE;
    memset(psi, 0, sizeof(cplx) * N);
    psi[x] = 1.0;
    return OR_OK;
}

/* Build stamp so that the Python wrapper can detect a stale shared object. */
int or_version(void) { return 3; }

/*
 * Plain CPU complex128 oracle for Pauli-rotation time evolution
 * (Miller et al., "phase2: Full-State Vector Simulation of Quantum Time
 * Evolution at Scale", arXiv:2504.17881).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke
 * check of the package entry file and the CPU-baseline leg of the benchmark
 * may load this library.  It shares no source, header, table or helper with
 * the CUDA library; both sides only consume the same seeded inputs.
 *
 * Everything is written for clarity, not speed: one loop per definition,
 * `double _Complex` amplitudes (the paper's own storage type, Methods,
 * "Mathematical model"), FP64 sums, no blocking, no fusion.
 * Compile with -ffp-contract=off so that every product is rounded as written.
 *
 * Built with -fopenmp, the element loops are shared among threads by plain
 * `omp parallel for` pragmas (or_set_threads; one thread by default).  Each
 * element is still computed by exactly the same expression: the scatter of
 * one rotation writes every output element once (k -> k XOR x is a
 * bijection), so threads never touch the same element.  Only the order of
 * the FP64 sums in or_overlap / or_norm2 depends on the thread count; with
 * one thread they run in index order.
 *
 * Conventions fixed by the paper:
 *   - qubit q (1-based, leftmost factor of the string) is bit q-1 of the
 *     basis-state index, least significant first (Results, "Software
 *     implementation": order of qubits from least to most significant);
 *   - a Pauli string is the bitmask pair (p1, p2) = (x, z): bit set in x iff
 *     the factor is X or Y, bit set in z iff it is Y or Z (Supplementary
 *     Methods, "Pauli-string bit representation"; worked example XIY -> (5, 4));
 *   - P|k> = omega_k |k XOR x>, omega_k a fourth root of unity.  The paper
 *     says omega comes from the number of Y factors (popcount of x AND z)
 *     and from the number of minus signs (popcount of z AND k).  Since
 *     Y = iXZ with Z acting first, omega_k = i^{popc(x&z)} (-1)^{popc(k&z)};
 *   - a rotation is exp(i phi P) = cos(phi) I + i sin(phi) P (Results,
 *     "Software implementation").
 *
 * Parity status: every function here is pinned by the "not gpu" tests
 * (dense Kronecker products and matrix exponentials, closed forms,
 * invariants, published SplitMix64 outputs).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------ threads */

/* Threads of the element loops (ignored without OpenMP).  Returns the
 * number in effect: 1 when the library was built without OpenMP. */
int or_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
    omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* 1 when built with OpenMP, else 0. */
int or_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ---------------------------------------------------------------- encoding */

/* Pauli string "XIY..." (leftmost character = qubit 1 = bit 0) -> (x, z).
 * Supplementary Methods, "Pauli-string bit representation".
 * Returns 0 on success, -1 on an unknown character or more than 64 factors. */
int or_pauli_from_string(const char *s, uint64_t *x, uint64_t *z)
{
    uint64_t xm = 0, zm = 0;
    int q = 0;
    for (; s[q] != '\0'; ++q) {
        if (q >= 64) return -1;
        uint64_t bit = (uint64_t)1 << q;
        switch (s[q]) {
        case 'I': break;
        case 'X': xm |= bit; break;
        case 'Y': xm |= bit; zm |= bit; break;
        case 'Z': zm |= bit; break;
        default: return -1;
        }
    }
    *x = xm;
    *z = zm;
    return 0;
}

static int popcount64(uint64_t v) { return __builtin_popcountll(v); }

/* i^m, m taken mod 4 */
static cplx i_pow(int m)
{
    switch (m & 3) {
    case 0: return 1.0;
    case 1: return I;
    case 2: return -1.0;
    default: return -I;
    }
}

/* omega_k with P|k> = omega_k |k ^ x>:  i^{#Y} * (-1)^{#(Y or Z acting on a 1 bit)}.
 * Supplementary Methods, "Pauli-string bit representation". */
static cplx omega(uint64_t x, uint64_t z, uint64_t k)
{
    cplx w = i_pow(popcount64(x & z));
    if (popcount64(k & z) & 1) w = -w;
    return w;
}

void or_pauli_phase(uint64_t x, uint64_t z, uint64_t k, double out[2])
{
    cplx w = omega(x, z, k);
    out[0] = creal(w);
    out[1] = cimag(w);
}

/* ------------------------------------------------------------- one rotation */

/* psi <- exp(i phi P) psi, P = (x, z), written as the scatter of the
 * definition exp(i phi P) = cos(phi) I + i sin(phi) P  (Results, "Software
 * implementation"):
 *     out[k]      = cos(phi) psi[k]                    for every k,
 *     out[k ^ x] += i sin(phi) omega_k psi[k]          for every k.
 * `tmp` is caller-provided scratch of 2^n amplitudes. */
int or_rotate(int n, cplx *psi, cplx *tmp, uint64_t x, uint64_t z, double phi)
{
    if (n < 1 || n > 40) return -1;
    uint64_t N = (uint64_t)1 << n;
    if ((x | z) >> n) return -1;
    double c = cos(phi), s = sin(phi);
#pragma omp parallel for schedule(static)
    for (uint64_t k = 0; k < N; ++k) tmp[k] = c * psi[k];
#pragma omp parallel for schedule(static)
    for (uint64_t k = 0; k < N; ++k) tmp[k ^ x] += (I * s) * omega(x, z, k) * psi[k];
#pragma omp parallel for schedule(static)
    for (uint64_t k = 0; k < N; ++k) psi[k] = tmp[k];
    return 0;
}

/* Apply a sequence: rotation 0 first, then 1, ... (the rightmost factor of a
 * product acts first; the sequence is given in application order). */
int or_apply(int n, cplx *psi, cplx *tmp, const uint64_t *x, const uint64_t *z,
             const double *phi, size_t count)
{
    for (size_t j = 0; j < count; ++j) {
        int rc = or_rotate(n, psi, tmp, x[j], z[j], phi[j]);
        if (rc) return rc;
    }
    return 0;
}

/* ----------------------------------------------------------- inner products */

/* <a|b> = sum_k conj(a[k]) b[k], summed in index order in FP64
 * (the signal g(t) of Methods, "Data analysis", Eq. 9). */
void or_overlap(int n, const cplx *a, const cplx *b, double out[2])
{
    uint64_t N = (uint64_t)1 << n;
    double re = 0.0, im = 0.0; /* the real and imaginary parts of the running complex sum */
#pragma omp parallel for schedule(static) reduction(+ : re, im)
    for (uint64_t k = 0; k < N; ++k) {
        cplx p = conj(a[k]) * b[k];
        re += creal(p);
        im += cimag(p);
    }
    out[0] = re;
    out[1] = im;
}

double or_norm2(int n, const cplx *a)
{
    uint64_t N = (uint64_t)1 << n;
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (uint64_t k = 0; k < N; ++k) acc += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return acc;
}

/* ------------------------------------------------------------ product formulas */

/* First-order Trotter (Methods, "Hamiltonian simulation", Eq. 3):
 *   exp(i t H) ~ ( prod_{l=1..L} exp(i delta h_l P_l) )^r,  delta = t / r,
 * with term l = 1 applied first in every step. */
int or_trotter(int n, cplx *psi, cplx *tmp, size_t L, const uint64_t *x, const uint64_t *z,
               const double *h, double t, uint32_t r)
{
    if (r == 0) return -1;
    double delta = t / (double)r;
    for (uint32_t step = 0; step < r; ++step)
        for (size_t l = 0; l < L; ++l) {
            int rc = or_rotate(n, psi, tmp, x[l], z[l], delta * h[l]);
            if (rc) return rc;
        }
    return 0;
}

/* Second-order (symmetric) product formula: each of r steps of delta = t/r
 * applies exp(i (delta/2) h_l P_l) for l = 1..L and then for l = L..1
 * (Methods: "This work uses the second-order variant"; the standard
 * symmetric splitting).  Written out factor by factor, without merging
 * the adjacent equal factors. */
int or_trotter2(int n, cplx *psi, cplx *tmp, size_t L, const uint64_t *x, const uint64_t *z,
                const double *h, double t, uint32_t r)
{
    if (r == 0) return -1;
    double half = 0.5 * (t / (double)r);
    for (uint32_t step = 0; step < r; ++step) {
        for (size_t l = 0; l < L; ++l) {
            int rc = or_rotate(n, psi, tmp, x[l], z[l], half * h[l]);
            if (rc) return rc;
        }
        for (size_t l = L; l-- > 0;) {
            int rc = or_rotate(n, psi, tmp, x[l], z[l], half * h[l]);
            if (rc) return rc;
        }
    }
    return 0;
}

/* SplitMix64 (Steele, Lea & Flood 2014): state += 0x9e3779b97f4a7c15, then
 * the published two-multiply finaliser.  Counter-based: the j-th output
 * (j = 1, 2, ...) depends only on seed + j * 0x9e3779b97f4a7c15. */
uint64_t or_splitmix64_next(uint64_t *state)
{
    uint64_t zz = (*state += 0x9e3779b97f4a7c15ULL);
    zz = (zz ^ (zz >> 30)) * 0xbf58476d1ce4e5b9ULL;
    zz = (zz ^ (zz >> 27)) * 0x94d049bb133111ebULL;
    return zz ^ (zz >> 31);
}

/* One draw: u = top 53 bits / 2^53 in [0, 1); return the smallest l with
 * cdf[l] > u * lambda, where cdf is the running FP64 sum of |h| in the
 * given order and lambda = cdf[L-1].  Linear scan, as written. */
static size_t draw_term(const double *cdf, size_t L, uint64_t *state)
{
    double u = (double)(or_splitmix64_next(state) >> 11) * 0x1.0p-53;
    double target = u * cdf[L - 1];
    for (size_t l = 0; l < L; ++l)
        if (cdf[l] > target) return l;
    return L - 1; /* unreachable: u < 1 */
}

static double *make_cdf(size_t L, const double *h, const size_t *members)
{
    double *cdf = (double *)malloc((L ? L : 1) * sizeof(double));
    if (!cdf) return NULL;
    double acc = 0.0;
    for (size_t l = 0; l < L; ++l) {
        acc += fabs(h[members ? members[l] : l]);
        cdf[l] = acc;
    }
    return cdf;
}

/* qDRIFT term indices (Campbell 2019, named in Methods, "Hamiltonian
 * simulation"): draws first .. first+count-1 of the sample stream for seed,
 * each term l drawn with probability |h_l| / lambda. */
int or_qdrift_indices(size_t L, const double *h, uint64_t seed, uint64_t first, uint64_t count,
                      uint64_t *idx_out)
{
    if (L == 0) return -1;
    double *cdf = make_cdf(L, h, NULL);
    if (!cdf) return -2;
    if (!(cdf[L - 1] > 0.0)) { free(cdf); return -1; }
    uint64_t state = seed + first * 0x9e3779b97f4a7c15ULL;
    for (uint64_t j = 0; j < count; ++j) idx_out[j] = draw_term(cdf, L, &state);
    free(cdf);
    return 0;
}

/* qDRIFT: N draws l_j, each applying exp(i sgn(h_{l_j}) (lambda t / N) P_{l_j}), in draw order. */
int or_qdrift(int n, cplx *psi, cplx *tmp, size_t L, const uint64_t *x, const uint64_t *z,
              const double *h, double t, uint64_t N, uint64_t seed)
{
    if (L == 0 || N == 0) return -1;
    double *cdf = make_cdf(L, h, NULL);
    if (!cdf) return -2;
    double lambda = cdf[L - 1];
    if (!(lambda > 0.0)) { free(cdf); return -1; }
    double tau = lambda * t / (double)N;
    uint64_t state = seed;
    for (uint64_t j = 0; j < N; ++j) {
        size_t l = draw_term(cdf, L, &state);
        double phi = h[l] > 0.0 ? tau : -tau;
        int rc = or_rotate(n, psi, tmp, x[l], z[l], phi);
        if (rc) { free(cdf); return rc; }
    }
    free(cdf);
    return 0;
}

/* Split of Eq. 5 (Methods, "Hamiltonian simulation"): the L_D terms of
 * largest |h| form H_D (ties broken by the lower index), the rest H_R.
 * Both parts keep the input order.  is_det[l] = 1 for l in H_D. */
int or_partial_split(size_t L, const double *h, size_t L_D, unsigned char *is_det)
{
    if (L_D > L) return -1;
    memset(is_det, 0, L);
    /* selection by repeated arg-max: plain and obviously correct */
    for (size_t taken = 0; taken < L_D; ++taken) {
        size_t best = L;
        for (size_t l = 0; l < L; ++l) {
            if (is_det[l]) continue;
            if (best == L || fabs(h[l]) > fabs(h[best])) best = l;
        }
        is_det[best] = 1;
    }
    return 0;
}

/* Partially randomised product formula, first-order reading of Eq. 5:
 * r steps of delta = t / r; each step applies every term of H_D as
 * exp(i delta h_l P_l) in input order, then Ns qDRIFT draws from H_R, each
 * exp(i sgn(h) (lambda_R delta / Ns) P).  One SplitMix64 stream (seeded
 * once) runs through all steps.  With L_D = L this is or_trotter; with
 * L_D = 0 and r = 1 it is or_qdrift with N = Ns. */
int or_partial(int n, cplx *psi, cplx *tmp, size_t L, const uint64_t *x, const uint64_t *z,
               const double *h, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed)
{
    if (r == 0 || L_D > L) return -1;
    unsigned char *is_det = (unsigned char *)malloc(L ? L : 1);
    size_t *rest = (size_t *)malloc((L ? L : 1) * sizeof(size_t));
    if (!is_det || !rest) { free(is_det); free(rest); return -2; }
    or_partial_split(L, h, L_D, is_det);
    size_t LR = 0;
    for (size_t l = 0; l < L; ++l)
        if (!is_det[l]) rest[LR++] = l;
    double *cdf = make_cdf(LR, h, rest);
    if (!cdf) { free(is_det); free(rest); return -2; }
    double lambda_R = LR ? cdf[LR - 1] : 0.0;
    double delta = t / (double)r;
    int sample = (LR > 0 && Ns > 0 && lambda_R > 0.0);
    double tau = sample ? lambda_R * delta / (double)Ns : 0.0;
    uint64_t state = seed;
    int rc = 0;
    for (uint32_t step = 0; step < r && !rc; ++step) {
        for (size_t l = 0; l < L && !rc; ++l)
            if (is_det[l]) rc = or_rotate(n, psi, tmp, x[l], z[l], delta * h[l]);
        if (!sample) continue;
        for (uint64_t j = 0; j < Ns && !rc; ++j) {
            size_t m = draw_term(cdf, LR, &state);
            size_t l = rest[m];
            rc = or_rotate(n, psi, tmp, x[l], z[l], h[l] > 0.0 ? tau : -tau);
        }
    }
    free(cdf);
    free(is_det);
    free(rest);
    return rc;
}

/* Second-order partially randomised step (the reading used here; the
 * paper states only that the randomised part takes twice the samples per
 * step at second order, Methods): per step of delta = t/r, the
 * deterministic terms forward with delta/2, then 2 Ns draws from H_R each
 * with angle sgn(h) lambda_R delta / (2 Ns), then the deterministic terms
 * backward with delta/2.  One SplitMix64 stream runs through all steps. */
int or_partial2(int n, cplx *psi, cplx *tmp, size_t L, const uint64_t *x, const uint64_t *z,
                const double *h, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed)
{
    if (r == 0 || L_D > L) return -1;
    unsigned char *is_det = (unsigned char *)malloc(L ? L : 1);
    size_t *rest = (size_t *)malloc((L ? L : 1) * sizeof(size_t));
    if (!is_det || !rest) { free(is_det); free(rest); return -2; }
    or_partial_split(L, h, L_D, is_det);
    size_t LR = 0;
    for (size_t l = 0; l < L; ++l)
        if (!is_det[l]) rest[LR++] = l;
    double *cdf = make_cdf(LR, h, rest);
    if (!cdf) { free(is_det); free(rest); return -2; }
    double lambda_R = LR ? cdf[LR - 1] : 0.0;
    double delta = t / (double)r;
    int sample = (LR > 0 && Ns > 0 && lambda_R > 0.0);
    double tau = sample ? lambda_R * delta / (double)(2 * Ns) : 0.0;
    uint64_t state = seed;
    int rc = 0;
    for (uint32_t step = 0; step < r && !rc; ++step) {
        for (size_t l = 0; l < L && !rc; ++l)
            if (is_det[l]) rc = or_rotate(n, psi, tmp, x[l], z[l], 0.5 * delta * h[l]);
        if (sample)
            for (uint64_t j = 0; j < 2 * Ns && !rc; ++j) {
                size_t m = draw_term(cdf, LR, &state);
                size_t l = rest[m];
                rc = or_rotate(n, psi, tmp, x[l], z[l], h[l] > 0.0 ? tau : -tau);
            }
        for (size_t l = L; l-- > 0 && !rc;)
            if (is_det[l]) rc = or_rotate(n, psi, tmp, x[l], z[l], 0.5 * delta * h[l]);
    }
    free(cdf);
    free(is_det);
    free(rest);
    return rc;
}

/* ------------------------------------------------- single amplitudes, any n */

/* Amplitude <k| U_R ... U_1 |psi0> for a sparse initial state (nnz basis
 * states idx0 with amplitudes amp0 as re/im pairs), by expanding the
 * definition of one rotation backwards:
 *   <k| exp(i phi P) |v> = cos(phi) <k|v> + i sin(phi) omega_{k^x} <k^x|v>
 * because P|k^x> = omega_{k^x}|k>.  Cost 2^(number of non-diagonal
 * rotations); meant for n up to 34 with short prefixes. */
static cplx sparse_lookup(size_t nnz, const uint64_t *idx0, const double *amp0, uint64_t k)
{
    for (size_t i = 0; i < nnz; ++i)
        if (idx0[i] == k) return amp0[2 * i] + I * amp0[2 * i + 1];
    return 0.0;
}

static cplx amp_rec(size_t level, uint64_t k, size_t nnz, const uint64_t *idx0, const double *amp0,
                    const uint64_t *x, const uint64_t *z, const double *cs, const double *sn)
{
    if (level == 0) return sparse_lookup(nnz, idx0, amp0, k);
    size_t j = level - 1;
    double c = cs[j], s = sn[j];
    uint64_t kp = k ^ x[j];
    if (kp == k) {
        cplx prev = amp_rec(j, k, nnz, idx0, amp0, x, z, cs, sn);
        return c * prev + (I * s) * omega(x[j], z[j], kp) * prev;
    }
    return c * amp_rec(j, k, nnz, idx0, amp0, x, z, cs, sn) +
           (I * s) * omega(x[j], z[j], kp) * amp_rec(j, kp, nnz, idx0, amp0, x, z, cs, sn);
}

int or_amplitudes_sparse(int n, size_t nnz, const uint64_t *idx0, const double *amp0,
                         const uint64_t *x, const uint64_t *z, const double *phi, size_t R,
                         size_t nk, const uint64_t *ks, double *out)
{
    if (n < 1 || n > 64) return -1;
    size_t nondiag = 0;
    for (size_t j = 0; j < R; ++j) nondiag += (x[j] != 0);
    if (nondiag > 26) return -1;
    /* cos and sin of every angle, once (the recursion visits each level many times) */
    double *cs = (double *)malloc((R ? R : 1) * sizeof(double));
    double *sn = (double *)malloc((R ? R : 1) * sizeof(double));
    if (!cs || !sn) { free(cs); free(sn); return -2; }
    for (size_t j = 0; j < R; ++j) {
        cs[j] = cos(phi[j]);
        sn[j] = sin(phi[j]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (size_t i = 0; i < nk; ++i) {
        cplx a = amp_rec(R, ks[i], nnz, idx0, amp0, x, z, cs, sn);
        out[2 * i] = creal(a);
        out[2 * i + 1] = cimag(a);
    }
    free(cs);
    free(sn);
    return 0;
}

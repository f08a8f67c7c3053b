/*
 * CPU oracle for the tall-and-skinny GEMM  C = alpha*A*B + beta*C0  (Eq. 1 of
 * "AutoTSMM", Li et al., arXiv 2208.08088; also the Output clause of its
 * Algorithm 1).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite,
 * the smoke check and the bench's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library: it reads the plain,
 * unpacked, column-major operands and evaluates the definition directly.
 *
 * Why the plain definition is the right oracle: the paper's method (packing,
 * cache blocking, per-thread panels; Section IV.A) only reorders the k-term
 * sums of Eq. 1, so the exact result it aims at is Eq. 1 itself.
 *
 * Conventions (the readings the paper leaves open, stated once):
 *   - column-major storage with explicit leading dimensions;
 *   - alpha and beta are applied exactly once (Eq. 1), not twice as a literal
 *     reading of Algorithm 1's COMPUTE would do;
 *   - alpha == 0: A and B are not read, C = beta*C0;
 *   - beta == 0: C0 is not read (may be NULL), C = alpha*A*B;
 *   - for the FP32 entry point alpha and beta are first rounded to float,
 *     exactly as the library does with its double-typed scalars.
 *
 * Outputs (both m x n column-major with leading dimension m, in double):
 *   Cref[i,j] = alpha * sum_p A[i,p]*B[p,j] + beta*C0[i,j]
 *   E[i,j]    = 4*k*u*( |alpha| * sum_p |A[i,p]|*|B[p,j]| + |beta|*|C0[i,j]| )
 * with u = 2^-24 (FP32) or 2^-53 (FP64): the componentwise acceptance bound,
 * Higham's gamma_k bound for a k-term dot product widened four times.
 *
 * FP32 entry point: products of two floats are exact in double and the
 * double sum adds at most k*2^-53*sum|A||B|, negligible next to E.
 *
 * FP64 entry point: the k-term dot product is the compensated "Dot2"
 * algorithm of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
 * Sci. Comput. 26(6), 2005): TwoProduct (via fma) and TwoSum error-free
 * transformations, accumulated in the order p = 0..k-1, so the result is as
 * accurate as if computed in twice the working precision and then rounded.
 * The final alpha*S + beta*C0 is a 3-term Dot2 of (alpha, alpha, beta) with
 * (S_hi, S_lo, C0).  This file must be compiled with -ffp-contract=off so the
 * compiler cannot fuse the TwoSum steps.
 *
 * Every sum runs over p = 0..k-1 in order for each (i, j), independent of
 * the thread count, so the oracle is deterministic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1
#define ORACLE_NO_MEM 2

#define ROW_BLOCK 512

/* ---- error-free transformations (Ogita, Rump & Oishi 2005, Alg. 3.1/3.3) -- */
static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

static int check_args(int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                      int64_t ldc, double alpha, double beta, const void *A, const void *B,
                      const void *C0, const void *Cref, const void *E) {
    if (m < 0 || n < 0 || k < 0) return ORACLE_BAD_ARG;
    if (m == 0 || n == 0) return ORACLE_OK;
    if (!Cref || !E) return ORACLE_BAD_ARG;
    if (alpha != 0.0 && k > 0) {
        if (!A || !B || lda < (m > 1 ? m : 1) || ldb < (k > 1 ? k : 1)) return ORACLE_BAD_ARG;
    }
    if (beta != 0.0) {
        if (!C0 || ldc < (m > 1 ? m : 1)) return ORACLE_BAD_ARG;
    }
    return ORACLE_OK;
}

/*
 * FP32 operands, FP64 accumulation.
 */
int oracle_tsmm_f32(int64_t m, int64_t n, int64_t k, double alpha_in, const float *A, int64_t lda,
                    const float *B, int64_t ldb, double beta_in, const float *C0, int64_t ldc,
                    double *Cref, double *E) {
    const double alpha = (double)(float)alpha_in;
    const double beta = (double)(float)beta_in;
    int rc = check_args(m, n, k, lda, ldb, ldc, alpha, beta, A, B, C0, Cref, E);
    if (rc != ORACLE_OK || m == 0 || n == 0) return rc;
    const double u = ldexp(1.0, -24);
    const int use_ab = (alpha != 0.0 && k > 0);
    const int64_t nblk = (m + ROW_BLOCK - 1) / ROW_BLOCK;
    int failed = 0;

#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (int64_t blk = 0; blk < nblk; ++blk) {
        const int64_t i0 = blk * ROW_BLOCK;
        const int64_t i1 = (i0 + ROW_BLOCK < m) ? i0 + ROW_BLOCK : m;
        const int64_t len = i1 - i0;
        double *S = (double *)malloc((size_t)len * sizeof(double));
        double *G = (double *)malloc((size_t)len * sizeof(double));
        if (!S || !G) {
            free(S);
            free(G);
            failed |= 1;
            continue;
        }
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t t = 0; t < len; ++t) { S[t] = 0.0; G[t] = 0.0; }
            if (use_ab) {
                for (int64_t p = 0; p < k; ++p) {
                    const double b = (double)B[p + j * ldb];
                    const float *a_col = A + p * lda + i0;
                    for (int64_t t = 0; t < len; ++t) {
                        const double prod = (double)a_col[t] * b; /* exact */
                        S[t] += prod;
                        G[t] += fabs(prod);
                    }
                }
            }
            for (int64_t t = 0; t < len; ++t) {
                const int64_t i = i0 + t;
                double c0 = 0.0;
                if (beta != 0.0) c0 = (double)C0[i + j * ldc];
                /* without the A*B term the result is beta*c0 itself (exact in
                   double, since beta and c0 are both floats), sign of zero kept */
                const double r = use_ab ? alpha * S[t] + beta * c0 : beta * c0;
                Cref[i + j * m] = r;
                E[i + j * m] = 4.0 * (double)k * u * (fabs(alpha) * G[t] + fabs(beta) * fabs(c0));
            }
        }
        free(S);
        free(G);
    }
    return failed ? ORACLE_NO_MEM : ORACLE_OK;
}

/*
 * FP64 operands, compensated (Dot2) accumulation.
 */
int oracle_tsmm_f64(int64_t m, int64_t n, int64_t k, double alpha, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double beta, const double *C0, int64_t ldc,
                    double *Cref, double *E) {
    int rc = check_args(m, n, k, lda, ldb, ldc, alpha, beta, A, B, C0, Cref, E);
    if (rc != ORACLE_OK || m == 0 || n == 0) return rc;
    const double u = ldexp(1.0, -53);
    const int use_ab = (alpha != 0.0 && k > 0);
    const int64_t nblk = (m + ROW_BLOCK - 1) / ROW_BLOCK;
    int failed = 0;

#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (int64_t blk = 0; blk < nblk; ++blk) {
        const int64_t i0 = blk * ROW_BLOCK;
        const int64_t i1 = (i0 + ROW_BLOCK < m) ? i0 + ROW_BLOCK : m;
        const int64_t len = i1 - i0;
        double *Sh = (double *)malloc((size_t)len * sizeof(double));
        double *Sl = (double *)malloc((size_t)len * sizeof(double));
        double *P = (double *)malloc((size_t)len * sizeof(double));
        double *G = (double *)malloc((size_t)len * sizeof(double));
        if (!Sh || !Sl || !P || !G) {
            free(Sh);
            free(Sl);
            free(P);
            free(G);
            failed |= 1;
            continue;
        }
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t t = 0; t < len; ++t) { Sh[t] = 0.0; Sl[t] = 0.0; P[t] = 0.0; G[t] = 0.0; }
            if (use_ab) {
                for (int64_t p = 0; p < k; ++p) {
                    const double b = B[p + j * ldb];
                    const double *a_col = A + p * lda + i0;
                    for (int64_t t = 0; t < len; ++t) {
                        double h, l, s, e;
                        two_prod(a_col[t], b, &h, &l);
                        two_sum(Sh[t], h, &s, &e);
                        Sh[t] = s;
                        Sl[t] += e + l;
                        P[t] += h;
                        G[t] += fabs(h);
                    }
                }
            }
            for (int64_t t = 0; t < len; ++t) {
                const int64_t i = i0 + t;
                double c0 = 0.0;
                if (beta != 0.0) c0 = C0[i + j * ldc];
                double r;
                /* Error-free transformations are undefined on infinities
                   (fma(inf, b, -inf) is NaN), so a non-finite plain result is
                   returned as IEEE arithmetic gives it: Inf or NaN inputs give
                   the same Inf/NaN in any summation order. */
                const double r_plain = use_ab ? alpha * P[t] + beta * c0 : beta * c0;
                if (!isfinite(r_plain)) {
                    r = r_plain;
                } else if (use_ab) {
                    /* Dot2 of (alpha, alpha, beta) . (Sh, Sl, c0) */
                    double p1, q1, p2, q2, p3, q3, s, e, tot;
                    two_prod(alpha, Sh[t], &p1, &q1);
                    two_prod(alpha, Sl[t], &p2, &q2);
                    two_prod(beta, c0, &p3, &q3);
                    two_sum(p1, p2, &s, &e);
                    tot = e + q1 + q2;
                    two_sum(s, p3, &s, &e);
                    tot += e + q3;
                    r = s + tot;
                } else {
                    r = beta * c0;
                }
                Cref[i + j * m] = r;
                E[i + j * m] = 4.0 * (double)k * u * (fabs(alpha) * G[t] + fabs(beta) * fabs(c0));
            }
        }
        free(Sh);
        free(Sl);
        free(P);
        free(G);
    }
    return failed ? ORACLE_NO_MEM : ORACLE_OK;
}

/* Number of threads an OpenMP parallel region would use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

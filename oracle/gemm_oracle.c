/*
 * CPU oracle for classical matrix multiplication C = A B (test infrastructure).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code with the CUDA library and is never on the
 * product path.
 *
 * What is computed is the plain definition of the product the paper studies
 * (Sec. 2.4: A is m x k, B is k x n, C is m x n; Sec. 5.1: every C element is
 * the chain of k partial sums c(i,j,t) = c(i,j,t-1) + a(i,t) b(t,j)).
 *
 *   oracle_gemm_naive   the partial-sum chain in the order t = 0..k-1, one
 *                       rounded multiply and one rounded add per step (built
 *                       with -ffp-contract=off so no fused multiply-add is
 *                       formed).
 *   oracle_gemm_dot2    the same sums evaluated with the compensated dot
 *                       product Dot2 of Ogita, Rump and Oishi ("Accurate sum
 *                       and dot product", SIAM J. Sci. Comput. 26(6), 2005,
 *                       Algorithm 5.3): TwoProduct via fma, TwoSum (Knuth).
 *                       The result is as accurate as if computed in twice the
 *                       working precision and then rounded.
 *   oracle_dot2_pairs   Dot2 of given row/column pairs (sampled entries of a
 *                       product too large for the full loop).
 *   oracle_freivalds    Freivalds' check (1977): r = C x - A (B x) for a given
 *                       vector x, both products in Dot2, plus the scale
 *                       |A| (|B| |x|) against which r is judged.
 *
 * All matrices are row-major with leading dimensions in elements.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

/* Error-free transformations (Ogita-Rump-Oishi 2005, Algorithms 3.1 and 3.3). */
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

/* Dot2 over x[i*incx], y[i*incy], i < n. */
static double dot2_strided(int64_t n, const double *x, int64_t incx, const double *y,
                           int64_t incy) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double p, ep, es;
    two_prod(x[i * incx], y[i * incy], &p, &ep);
    two_sum(s, p, &s, &es);
    c += es + ep;
  }
  return s + c;
}

void oracle_gemm_naive(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                       const double *B, int64_t ldb, double *C, int64_t ldc) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double c = 0.0;
      for (int64_t t = 0; t < k; ++t) {
        double prod = A[i * lda + t] * B[t * ldb + j];
        c = c + prod;
      }
      C[i * ldc + j] = c;
    }
}

void oracle_gemm_dot2(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                      const double *B, int64_t ldb, double *C, int64_t ldc) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      C[i * ldc + j] = dot2_strided(k, A + i * lda, 1, B + j, ldb);
}

/* out[p] = Dot2(arows[p, :], bcols[p, :]) for p < count; both arrays are
 * count x k row-major (bcols holds columns of B laid out as rows). */
void oracle_dot2_pairs(int64_t count, int64_t k, const double *arows, const double *bcols,
                       double *out) {
  for (int64_t p = 0; p < count; ++p)
    out[p] = dot2_strided(k, arows + p * k, 1, bcols + p * k, 1);
}

/* r = C x - A (B x) and scale = |A| (|B| |x|), both of length m. */
void oracle_freivalds(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                      const double *B, int64_t ldb, const double *C, int64_t ldc,
                      const double *x, double *bx, double *absbx, double *r, double *scale) {
  for (int64_t t = 0; t < k; ++t) {
    bx[t] = dot2_strided(n, B + t * ldb, 1, x, 1);
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += fabs(B[t * ldb + j]) * fabs(x[j]);
    absbx[t] = s;
  }
  for (int64_t i = 0; i < m; ++i) {
    /* C x - A (B x) as one compensated dot product of length n + k. */
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double p, ep, es;
      two_prod(C[i * ldc + j], x[j], &p, &ep);
      two_sum(s, p, &s, &es);
      c += es + ep;
    }
    for (int64_t t = 0; t < k; ++t) {
      double p, ep, es;
      two_prod(-A[i * lda + t], bx[t], &p, &ep);
      two_sum(s, p, &s, &es);
      c += es + ep;
    }
    r[i] = s + c;
    double a = 0.0;
    for (int64_t t = 0; t < k; ++t) a += fabs(A[i * lda + t]) * absbx[t];
    scale[i] = a;
  }
}

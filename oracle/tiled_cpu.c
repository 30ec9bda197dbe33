/*
 * Test infrastructure only: the benchmark's all-core CPU timing beside the GPU
 * results.  Never on the product path; no code shared with the CUDA library.
 *
 * C = A B under the sequential schedule that Sec. 5.2 arrives at: one
 * processor's fast memory holds a near-square a x b block of C (the tile shape
 * maximising ab / (a + b) subject to ab + a + 1 <= S, eq. aopt/bopt and the
 * optimisation problem it solves), every entry of the block is finished while
 * it stays resident, and only then is the block written back.  The loop
 * structure is this file's own: blocks of C are spread over OpenMP threads;
 * inside a block, k is walked in panels of KC; the KC rows of B a panel needs
 * are first packed into a contiguous KC x w buffer, then each row i of the
 * block takes the panel's KC rank-1 contributions A[i, t] B[t, :] in turn.
 *
 * Every entry receives its products one at a time in the order t = 0..k-1 (one
 * rounded multiply and one rounded add each: built with -ffp-contract=off), so
 * each is the partial-sum chain of oracle_gemm_naive in gemm_oracle.c, bit for
 * bit -- which the tests check.
 *
 * Row-major, leading dimensions in elements.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { KC = 64 };  /* k panel of one packing pass */

/* Returns the number of threads used, or -1 when a block buffer cannot be allocated. */
int tiled_gemm(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B,
               int64_t ldb, double *C, int64_t ldc, int64_t a, int64_t b, int threads) {
  if (a < 1 || b < 1) return -1;
  const int64_t rows_of_blocks = (m + a - 1) / a, cols_of_blocks = (n + b - 1) / b;
  const int64_t blocks = rows_of_blocks * cols_of_blocks;
  int used = 1;
  int failed = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel reduction(| : failed)
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
    double *acc = (double *)malloc((size_t)(a * b) * sizeof(double));   /* the resident block */
    double *panel = (double *)malloc((size_t)(KC * b) * sizeof(double)); /* packed rows of B */
    if (!acc || !panel) failed = 1;
#pragma omp for schedule(dynamic, 1)
    for (int64_t blk = 0; blk < blocks; ++blk) {
      if (!acc || !panel) continue;
      const int64_t r0 = (blk / cols_of_blocks) * a, c0 = (blk % cols_of_blocks) * b;
      const int64_t h = m - r0 < a ? m - r0 : a;
      const int64_t w = n - c0 < b ? n - c0 : b;
      memset(acc, 0, (size_t)(h * w) * sizeof(double));
      for (int64_t t0 = 0; t0 < k; t0 += KC) {
        const int64_t kc = k - t0 < KC ? k - t0 : KC;
        for (int64_t u = 0; u < kc; ++u)
          memcpy(panel + u * w, B + (t0 + u) * ldb + c0, (size_t)w * sizeof(double));
        for (int64_t i = 0; i < h; ++i) {
          const double *arow = A + (r0 + i) * lda + t0;
          double *crow = acc + i * w;
          for (int64_t u = 0; u < kc; ++u) {
            const double x = arow[u];
            const double *brow = panel + u * w;
            for (int64_t j = 0; j < w; ++j) crow[j] = crow[j] + x * brow[j];
          }
        }
      }
      for (int64_t i = 0; i < h; ++i)
        memcpy(C + (r0 + i) * ldc + c0, acc + i * w, (size_t)w * sizeof(double));
    }
    free(acc);
    free(panel);
  }
  return failed ? -1 : used;
}

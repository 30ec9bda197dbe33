/*
 * The paper's sequential schedule (Listing 1, Sec. 5.2) on the host cores, for
 * the benchmark's CPU timing beside the GPU results (test infrastructure; never
 * on the product path, no code shared with the CUDA library).
 *
 * C is cut into a x b tiles (0-based, half-open, ragged last tiles).  Each tile
 * is one processor's resident block of fast memory: it is zeroed, then for
 * t = 0..k-1 the column segment A[i0:i1, t] and the row segment B[t, j0:j1]
 * are read and their outer product is added (one rounded multiply and one
 * rounded add per element: built with -ffp-contract=off), and the finished
 * tile is written once.  Every entry is therefore the partial-sum chain in the
 * order t = 0..k-1 -- bit-identical to oracle_gemm_naive in gemm_oracle.c,
 * which the tests check.  Tiles are distributed over OpenMP threads.
 *
 * Row-major, leading dimensions in elements.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Returns the number of threads used, or -1 when a tile buffer cannot be allocated. */
int listing1_gemm(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *C, int64_t ldc, int64_t a, int64_t b,
                  int threads) {
  if (a < 1 || b < 1) return -1;
  const int64_t mt = (m + a - 1) / a, nt = (n + b - 1) / b;
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
    double *tile = (double *)malloc((size_t)(a * b) * sizeof(double));
    if (!tile) failed = 1;
#pragma omp for schedule(dynamic, 1)
    for (int64_t q = 0; q < mt * nt; ++q) {
      if (!tile) continue;
      const int64_t i0 = (q / nt) * a, j0 = (q % nt) * b;
      const int64_t h = m - i0 < a ? m - i0 : a, w = n - j0 < b ? n - j0 : b;
      memset(tile, 0, (size_t)(h * w) * sizeof(double));
      for (int64_t t = 0; t < k; ++t) {
        const double *brow = B + t * ldb + j0;
        for (int64_t i = 0; i < h; ++i) {
          const double x = A[(i0 + i) * lda + t];
          double *c = tile + i * w;
          for (int64_t j = 0; j < w; ++j) c[j] = c[j] + x * brow[j];
        }
      }
      for (int64_t i = 0; i < h; ++i) memcpy(C + (i0 + i) * ldc + j0, tile + i * w,
                                             (size_t)w * sizeof(double));
    }
    free(tile);
  }
  return failed ? -1 : used;
}

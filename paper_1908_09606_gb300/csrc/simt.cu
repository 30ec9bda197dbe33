// K-F64 / K-F32: C-stationary tile kernels on the FMA pipes, and the split-k
// Reduce (Alg. 1 Reduce).
//
// Each CTA is one processor of the schedule: it walks the work units of its
// local domain (schedule.h).  For one unit the tile_m x tile_n C tile stays in
// registers (8 x 8 or 4 x 4 per thread) while A-column and B-row panels of
// k_block outer products stream through a double-buffered shared-memory ring
// -- the rank-1-update order of Listing 1 with a k_block-deep step (Alg. 1's
// step size s).  The next panel pair is fetched into registers while the
// current one is multiplied (the overlap of Sec. 7.3).
//
// GB300 has a narrow FP64 pipe, so K-F64 is bound by FP64 FMA issue; its
// global loads are plain (any alignment / leading dimension is accepted).
#include <cuda_runtime.h>

#include "internal.h"

namespace cosma {
namespace {

template <typename T>
struct VecW {
  static constexpr int V = 16 / sizeof(T);  // elements per 16-byte shared-memory access
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256)
simt_gemm_kernel(GemmArgs g, Sched s, T* partial) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  static_assert(BN / TN == 16 && BM / TM == 16, "16 x 16 thread grid");
  constexpr int V = VecW<T>::V;
  constexpr int A_PER = BM * BK / 256;
  constexpr int B_PER = BK * BN / 256;
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];

  const T* __restrict__ A = static_cast<const T*>(g.A);
  const T* __restrict__ B = static_cast<const T*>(g.B);
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int cta = blockIdx.x;
  const int64_t nunits = units_of_cta(s, cta);

  for (int64_t ui = 0; ui < nunits; ++ui) {
    const Unit u = unit_of_cta(s, cta, ui);
    const int64_t row0 = u.tile_row * BM, col0 = u.tile_col * BN;
    const int64_t kbeg = u.kb0 * (int64_t)s.k_block;
    const int64_t kend = min(u.kb1 * (int64_t)s.k_block, g.k);
    const int64_t nsteps = (kend - kbeg + BK - 1) / BK;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    T ra[A_PER], rb[B_PER];
    auto fetch = [&](int64_t k0) {
#pragma unroll
      for (int e = 0; e < A_PER; ++e) {
        const int idx = tid + e * 256;
        const int r = idx / BK, kk = idx % BK;
        const int64_t gr = row0 + r, gk = k0 + kk;
        ra[e] = (gr < g.m && gk < kend) ? A[gr * g.lda + gk] : T(0);
      }
#pragma unroll
      for (int e = 0; e < B_PER; ++e) {
        const int idx = tid + e * 256;
        const int kk = idx / BN, c = idx % BN;
        const int64_t gk = k0 + kk, gc = col0 + c;
        rb[e] = (gk < kend && gc < g.n) ? B[gk * g.ldb + gc] : T(0);
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int e = 0; e < A_PER; ++e) {
        const int idx = tid + e * 256;
        As[buf][idx % BK][idx / BK] = ra[e];
      }
#pragma unroll
      for (int e = 0; e < B_PER; ++e) {
        const int idx = tid + e * 256;
        Bs[buf][idx / BN][idx % BN] = rb[e];
      }
    };

    __syncthreads();  // previous unit's readers are done with the ring
    if (nsteps > 0) {
      fetch(kbeg);
      stash(0);
    }
    __syncthreads();
    for (int64_t st = 0; st < nsteps; ++st) {
      const int buf = (int)(st & 1);
      if (st + 1 < nsteps) fetch(kbeg + (st + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][(j / V) * (16 * V) + tx * V + (j % V)];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (st + 1 < nsteps) stash(buf ^ 1);
      __syncthreads();
    }

    // Epilogue: the C tile (or this k slice's partial) leaves fast memory.
    T* dst;
    int64_t ld;
    if (s.pk > 1) {
      dst = partial + (int64_t)u.ks * g.m * g.n;
      ld = g.n;
    } else {
      dst = static_cast<T*>(g.C);
      ld = g.ldc;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t r = row0 + ty * TM + i;
      if (r >= g.m) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t c = col0 + (j / V) * (16 * V) + tx * V + (j % V);
        if (c < g.n) dst[r * ld + c] = acc[i][j];
      }
    }
  }
}

// Reduce over the k dimension of the grid: C = sum_{ks = 0}^{pk-1} P[ks], in
// that fixed order, so the result does not depend on scheduling.
template <typename T>
__global__ void reduce_kernel(int64_t m, int64_t n, int pk, const T* __restrict__ partial,
                              T* __restrict__ C, int64_t ldc) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = partial[e];
    for (int q = 1; q < pk; ++q) acc += partial[(int64_t)q * total + e];
    const int64_t r = e / n, c = e - r * n;
    C[r * ldc + c] = acc;
  }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
int launch_tile(const GemmArgs& g, const Sched& s, void* partial, cudaStream_t st) {
  simt_gemm_kernel<T, BM, BN, BK, TM, TN>
      <<<s.ctas, 256, 0, st>>>(g, s, static_cast<T*>(partial));
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace

int launch_simt(int dtype, const GemmArgs& g, const Sched& s, void* partial, int* status,
                cudaStream_t st) {
  (void)status;
  if (dtype == COSMA_F64) {
    if (s.tile_m == 128) return launch_tile<double, 128, 128, 8, 8, 8>(g, s, partial, st);
    return launch_tile<double, 64, 64, 8, 4, 4>(g, s, partial, st);
  }
  if (s.tile_m == 128) return launch_tile<float, 128, 128, 16, 8, 8>(g, s, partial, st);
  return launch_tile<float, 64, 64, 16, 4, 4>(g, s, partial, st);
}

int launch_reduce(int dtype, const GemmArgs& g, int pk, const void* partial, cudaStream_t st) {
  const int64_t total = g.m * g.n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (dtype == COSMA_F64)
    reduce_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(
        g.m, g.n, pk, static_cast<const double*>(partial), static_cast<double*>(g.C), g.ldc);
  else
    reduce_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(
        g.m, g.n, pk, static_cast<const float*>(partial), static_cast<float*>(g.C), g.ldc);
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace cosma

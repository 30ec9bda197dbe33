// One C-stationary tile on the FMA pipes (shared by K-F64/K-F32 and the
// grouped FP32 kernel).  The tile_m x tile_n C tile stays in registers while
// k_block-deep A and B panels stream through a double-buffered shared-memory
// ring, the next panel pair prefetched into registers during the multiply.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cosma {

template <typename T>
struct VecW {
  static constexpr int V = 16 / sizeof(T);  // elements per 16-byte shared-memory access
};

template <typename T, int BM, int BN, int BK>
struct SimtSmem {
  T As[2][BK][BM];
  T Bs[2][BK][BN];
};

// Value stored for one C entry: alpha acc + beta c, with c read only when beta != 0.
template <typename T>
__device__ __forceinline__ void store_ab(T* p, T acc, T alpha, T beta) {
  T v = alpha == T(1) ? acc : alpha * acc;
  if (beta != T(0)) v = fma(beta, *p, v);
  *p = v;
}

// dst[(row0 + i) * ld + col0 + j] = alpha sum_{t in [kbeg, kend)} A[row0+i][t] B[t][col0+j]
//                                   (+ beta dst[...] when beta != 0)
template <typename T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void simt_tile(const T* __restrict__ A, int64_t lda,
                                          const T* __restrict__ B, int64_t ldb, T* dst, int64_t ld,
                                          int64_t m, int64_t n, int64_t row0, int64_t col0,
                                          int64_t kbeg, int64_t kend,
                                          SimtSmem<T, BM, BN, BK>& sm, T alpha = T(1),
                                          T beta = T(0)) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  static_assert(BN / TN == 16 && BM / TM == 16, "16 x 16 thread grid");
  constexpr int V = VecW<T>::V;
  constexpr int A_PER = BM * BK / 256;
  constexpr int B_PER = BK * BN / 256;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
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
      ra[e] = (gr < m && gk < kend) ? A[gr * lda + gk] : T(0);
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = tid + e * 256;
      const int kk = idx / BN, c = idx % BN;
      const int64_t gk = k0 + kk, gc = col0 + c;
      rb[e] = (gk < kend && gc < n) ? B[gk * ldb + gc] : T(0);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int idx = tid + e * 256;
      sm.As[buf][idx % BK][idx / BK] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = tid + e * 256;
      sm.Bs[buf][idx / BN][idx % BN] = rb[e];
    }
  };

  __syncthreads();  // previous tile's readers are done with the ring
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
      for (int i = 0; i < TM; ++i) a[i] = sm.As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = sm.Bs[buf][kk][(j / V) * (16 * V) + tx * V + (j % V)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (st + 1 < nsteps) stash(buf ^ 1);
    __syncthreads();
  }

  // Epilogue: the C tile (or a k slice's partial) leaves fast memory.
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t r = row0 + ty * TM + i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t c = col0 + (j / V) * (16 * V) + tx * V + (j % V);
      if (c < n) store_ab(&dst[r * ld + c], acc[i][j], alpha, beta);
    }
  }
}

}  // namespace cosma

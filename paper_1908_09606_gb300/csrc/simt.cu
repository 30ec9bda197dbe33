// K-F64 / K-F32: C-stationary tile kernels on the FMA pipes, and the split-k
// Reduce (Alg. 1 Reduce).
//
// Each CTA is one processor of the schedule: it walks the work units of its
// local domain (schedule.h).  For one unit the tile_m x tile_n C tile stays in
// registers (8 x 8 or 4 x 4 per thread) while A-column and B-row panels of
// k_block outer products stream through a shared-memory ring -- the
// rank-1-update order of Listing 1 with a k_block-deep step (Alg. 1's step
// size s).  K-F64 fetches the next panel pair into registers while the current
// one is multiplied; K-F32 keeps four panels in flight with cp.async
// (simt_f32.cuh); both overlap loads with multiplies as in Sec. 7.3.
//
// GB300 has a narrow FP64 pipe, so K-F64 is bound by FP64 FMA issue; its
// global loads are plain (any alignment / leading dimension is accepted).
#include <cuda_runtime.h>

#include "internal.h"
#include "simt_tile.cuh"
#include "simt_f32.cuh"

namespace cosma {
namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256)
simt_gemm_kernel(GemmArgs g, Sched s, T* partial) {
  __shared__ __align__(16) SimtSmem<T, BM, BN, BK> sm;
  const T* A = static_cast<const T*>(g.A);
  const T* B = static_cast<const T*>(g.B);
  const int cta = blockIdx.x;
  const int64_t nunits = units_of_cta(s, cta);
  for (int64_t ui = 0; ui < nunits; ++ui) {
    const Unit u = unit_of_cta(s, cta, ui);
    T* dst;
    int64_t ld;
    if (s.pk > 1) {
      dst = partial + (int64_t)u.ks * g.m * g.n;
      ld = g.n;
    } else {
      dst = static_cast<T*>(g.C);
      ld = g.ldc;
    }
    // split-k partials are raw sums; the Reduce applies alpha and beta
    const T al = s.pk > 1 ? T(1) : (T)g.alpha, be = s.pk > 1 ? T(0) : (T)g.beta;
    simt_tile<T, BM, BN, BK, TM, TN>(A, g.lda, B, g.ldb, dst, ld, g.m, g.n, u.tile_row * BM,
                                     u.tile_col * BN, u.kb0 * (int64_t)s.k_block,
                                     min(u.kb1 * (int64_t)s.k_block, g.k), sm, al, be);
  }
}

// K-F32: the cp.async multi-stage tile of simt_f32.cuh (BM x 128, 2 BM threads).
template <int BM, int VEC, int BN = F32_BN>
__global__ void __launch_bounds__(f32_threads<BM>(), 1)
simt_f32_kernel(GemmArgs g, Sched s, float* partial, int vec_c) {
  extern __shared__ __align__(16) uint8_t f32_smem[];
  F32Smem<BM, BN>& sm = *reinterpret_cast<F32Smem<BM, BN>*>(f32_smem);
  const float* A = static_cast<const float*>(g.A);
  const float* B = static_cast<const float*>(g.B);
  const int cta = blockIdx.x;
  const int64_t nunits = units_of_cta(s, cta);
  for (int64_t ui = 0; ui < nunits; ++ui) {
    const Unit u = unit_of_cta(s, cta, ui);
    float* dst;
    int64_t ld;
    bool vec;
    if (s.pk > 1) {
      dst = partial + (int64_t)u.ks * g.m * g.n;
      ld = g.n;
      vec = (g.n & 3) == 0;
    } else {
      dst = static_cast<float*>(g.C);
      ld = g.ldc;
      vec = vec_c != 0;
    }
    const float al = s.pk > 1 ? 1.f : (float)g.alpha, be = s.pk > 1 ? 0.f : (float)g.beta;
    f32_tile<BM, VEC, BN>(A, g.lda, B, g.ldb, dst, ld, g.m, g.n, u.tile_row * BM,
                          u.tile_col * BN, u.kb0 * (int64_t)s.k_block,
                          min(u.kb1 * (int64_t)s.k_block, g.k), vec, sm, al, be);
  }
}

// Reduce over the k dimension of the grid: C = alpha sum_{ks = 0}^{pk-1} P[ks]
// (+ beta C), the sum in that fixed order, so the result does not depend on
// scheduling.
template <typename T>
__global__ void reduce_kernel(int64_t m, int64_t n, int pk, const T* __restrict__ partial,
                              T* __restrict__ C, int64_t ldc, T alpha, T beta) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = partial[e];
    for (int q = 1; q < pk; ++q) acc += partial[(int64_t)q * total + e];
    const int64_t r = e / n, c = e - r * n;
    store_ab(&C[r * ldc + c], acc, alpha, beta);
  }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
int launch_tile(const GemmArgs& g, const Sched& s, void* partial, cudaStream_t st) {
  prof_mark(st, true);
  simt_gemm_kernel<T, BM, BN, BK, TM, TN>
      <<<s.ctas, 256, 0, st>>>(g, s, static_cast<T*>(partial));
  prof_mark(st, false);
  count_launch();
  return (int)cudaGetLastError();
}

// C = beta C over m x n (beta == 0: zeros, C not read).
template <typename T>
__global__ void scale_kernel(int64_t m, int64_t n, T* __restrict__ C, int64_t ldc, T beta) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, c = e - r * n;
    T* p = C + r * ldc + c;
    *p = beta == T(0) ? T(0) : beta * *p;
  }
}

// dst[j][i] = src[i][j] for a rows x cols src; 32 x 32 tiles through shared memory.
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ src, int64_t rows, int64_t cols,
                                 int64_t ld_src, T* __restrict__ dst, int64_t ld_dst) {
  __shared__ T tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = src[r * ld_src + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ld_dst + r] = tile[threadIdx.x][i];
  }
}

}  // namespace

int launch_scale(int dtype, const GemmArgs& g, cudaStream_t st) {
  const int64_t total = g.m * g.n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) return 0;
  if (dtype == COSMA_F32 || dtype == COSMA_BF16 || dtype == COSMA_F32_EMU_TF32)
    scale_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(g.m, g.n, static_cast<float*>(g.C),
                                                          g.ldc, (float)g.beta);
  else
    scale_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(g.m, g.n, static_cast<double*>(g.C),
                                                           g.ldc, g.beta);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_transpose(int elem_bytes, const void* src, int64_t rows, int64_t cols, int64_t ld_src,
                     void* dst, int64_t ld_dst, cudaStream_t st) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  if ((rows + 31) / 32 > 65535) return COSMA_ERR_UNSUPPORTED;
  if (elem_bytes == 8)
    transpose_kernel<double><<<grid, dim3(32, 8), 0, st>>>(static_cast<const double*>(src), rows,
                                                           cols, ld_src, static_cast<double*>(dst),
                                                           ld_dst);
  else
    transpose_kernel<float><<<grid, dim3(32, 8), 0, st>>>(static_cast<const float*>(src), rows,
                                                          cols, ld_src, static_cast<float*>(dst),
                                                          ld_dst);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_simt(int dtype, const GemmArgs& g, const Sched& s, void* partial, int* status,
                cudaStream_t st) {
  (void)status;
  if (dtype == COSMA_F64) {
    if (s.tile_m == 128) return launch_tile<double, 128, 128, 8, 8, 8>(g, s, partial, st);
    return launch_tile<double, 64, 64, 8, 4, 4>(g, s, partial, st);
  }
  const bool wide = s.tile_m == 128 && s.tile_n == 256;
  if (!wide && ((s.tile_m != 128 && s.tile_m != 256) || s.tile_n != F32_BN))
    return COSMA_ERR_INVALID_ARG;
  if (s.k_block % F32_BK) return COSMA_ERR_INVALID_ARG;
  const bool vec_ab = (reinterpret_cast<uintptr_t>(g.A) & 15) == 0 && (g.lda & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(g.B) & 15) == 0 && (g.ldb & 3) == 0;
  const int vec_c = (reinterpret_cast<uintptr_t>(g.C) & 15) == 0 && (g.ldc & 3) == 0;
  void (*kern)(GemmArgs, Sched, float*, int);
  int threads, smem;
  if (wide) {
    kern = vec_ab ? simt_f32_kernel<128, 4, 256> : simt_f32_kernel<128, 1, 256>;
    threads = f32_threads<128>();
    smem = (int)sizeof(F32Smem<128, 256>);
  } else if (s.tile_m == 256) {
    kern = vec_ab ? simt_f32_kernel<256, 4> : simt_f32_kernel<256, 1>;
    threads = f32_threads<256>();
    smem = (int)sizeof(F32Smem<256>);
  } else {
    kern = vec_ab ? simt_f32_kernel<128, 4> : simt_f32_kernel<128, 1>;
    threads = f32_threads<128>();
    smem = (int)sizeof(F32Smem<128>);
  }
  const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return (int)attr;
  prof_mark(st, true);
  kern<<<s.ctas, threads, smem, st>>>(g, s, static_cast<float*>(partial), vec_c);
  prof_mark(st, false);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_reduce(int dtype, const GemmArgs& g, int pk, const void* partial, cudaStream_t st) {
  const int64_t total = g.m * g.n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (dtype == COSMA_F64 || dtype == COSMA_F64_EMU_BF16)
    reduce_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(
        g.m, g.n, pk, static_cast<const double*>(partial), static_cast<double*>(g.C), g.ldc,
        g.alpha, g.beta);
  else
    reduce_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(
        g.m, g.n, pk, static_cast<const float*>(partial), static_cast<float*>(g.C), g.ldc,
        (float)g.alpha, (float)g.beta);
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace cosma

// Complex products (cosma_zgemm: double, cosma_cgemm: single):
// C = alpha op(A) op(B) + beta C over interleaved (re, im) storage, run as four
// real products on a real engine of the same precision -- the "4M" form:
//   Tr = Ar Br - Ai Bi,   Ti = Ar Bi + Ai Br,   C = alpha (Tr + i Ti) + beta C.
// op is the identity, the transpose, or the conjugate transpose; a transposed
// operand is stored transposed (A as k x m, B as n x k) and split into planar
// real and imaginary parts in that orientation (the imaginary part negated for a
// conjugate transpose), so the real products take it through their own
// transposed-operand paths.  Not in the paper; its ScaLAPACK interface carries
// the complex P?GEMM variants as well.
#include <cuda_runtime.h>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cosma {

namespace {

constexpr int kMaxDevices = 16;

struct ComplexState {
  void* stage = nullptr;
  size_t stage_bytes = 0;
  bool captured = false;       // stage is recorded in a captured graph
  std::vector<void*> retired;  // captured stages given up on growth; freed at finalize
};

std::mutex g_cplx_mu;
ComplexState g_cplx[kMaxDevices];

inline int64_t rup(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

// re / im (rows x cols, ld cols) from interleaved src (ld_src complex elements);
// im negated when conj.
template <class R>
__global__ void split_complex_kernel(const typename Cplx<R>::T* __restrict__ src, int64_t rows,
                                     int64_t cols, int64_t ld_src, R* __restrict__ re,
                                     R* __restrict__ im, int conj) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    const typename Cplx<R>::T v = src[r * ld_src + c];
    re[e] = v.x;
    im[e] = conj ? -v.y : v.y;
  }
}

// C = alpha (Tr + i Ti) + beta C (C read only when beta != 0), in R.
template <class R>
__global__ void combine_complex_kernel(int64_t m, int64_t n, const R* __restrict__ tr,
                                       const R* __restrict__ ti,
                                       typename Cplx<R>::T* __restrict__ C, int64_t ldc, R ar,
                                       R ai, R br, R bi) {
  const int64_t total = m * n;
  const bool read_c = br != R(0) || bi != R(0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, c = e - r * n;
    const R x = tr[e], y = ti[e];
    typename Cplx<R>::T out;
    out.x = ar * x - ai * y;
    out.y = ar * y + ai * x;
    if (read_c) {
      const typename Cplx<R>::T v = C[r * ldc + c];
      out.x += br * v.x - bi * v.y;
      out.y += br * v.y + bi * v.x;
    }
    C[r * ldc + c] = out;
  }
}

unsigned grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

void complex_release(int dev) {
  std::lock_guard<std::mutex> lock(g_cplx_mu);
  if (dev < 0 || dev >= kMaxDevices) return;
  if (g_cplx[dev].stage) cudaFree(g_cplx[dev].stage);
  for (void* p : g_cplx[dev].retired) cudaFree(p);
  g_cplx[dev] = ComplexState{};
}

}  // namespace cosma

namespace cosma {
namespace {

// Both precisions: R the real type, engine a real dtype of that precision.
template <class R>
int complex_gemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k, const R* alpha,
                 const void* A, int64_t lda, const void* B, int64_t ldb, const R* beta, void* C,
                 int64_t ldc, int engine, void* stream) {
  using C2 = typename Cplx<R>::T;
  const uintptr_t amask = sizeof(C2) - 1;
  if (op_a < 0 || op_a > 2 || op_b < 0 || op_b > 2 || !alpha || !beta) return COSMA_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0) return COSMA_ERR_INVALID_ARG;
  const int ta = op_a != 0, tb = op_b != 0;
  const int64_t a_rows = ta ? k : m, a_cols = ta ? m : k;
  const int64_t b_rows = tb ? n : k, b_cols = tb ? k : n;
  if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1) ||
      ldc < (n > 1 ? n : 1))
    return COSMA_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return COSMA_OK;
  if (k_supported(engine, k) != COSMA_OK) return COSMA_ERR_UNSUPPORTED;  // before any staging
  if (!C || (reinterpret_cast<uintptr_t>(C) & amask) || !on_device(C)) return COSMA_ERR_INVALID_ARG;
  const bool no_ab = k == 0 || (alpha[0] == R(0) && alpha[1] == R(0));
  if (!no_ab && (!A || !B || (reinterpret_cast<uintptr_t>(A) & amask) ||
                 (reinterpret_cast<uintptr_t>(B) & amask) || !on_device(A) || !on_device(B)))
    return COSMA_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return COSMA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_cplx_mu);
  ComplexState& cs = g_cplx[dev];

  // staging: Ar, Ai (a_rows x a_cols), Br, Bi (b_rows x b_cols), Tr, Ti (m x n)
  const int64_t kk = no_ab ? 0 : k;
  const int64_t w = (int64_t)sizeof(R);
  const size_t a_b = (size_t)rup(a_rows * a_cols * w * (kk > 0), 256);
  const size_t b_b = (size_t)rup(b_rows * b_cols * w * (kk > 0), 256);
  const size_t t_b = (size_t)rup(m * n * w, 256);
  const size_t need = 2 * a_b + 2 * b_b + 2 * t_b;
  const bool cap = capturing(st);
  if (cs.stage_bytes < need) {
    if (cap) return COSMA_ERR_NO_WORKSPACE;
    if (cs.stage) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return COSMA_ERR_CUDA;
      if (cs.captured) cs.retired.push_back(cs.stage);  // a graph may still read it
      else cudaFree(cs.stage);
      cs.stage = nullptr;
      cs.stage_bytes = 0;
      cs.captured = false;
    }
    const size_t want = (need + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    if (cudaMalloc(&cs.stage, want) != cudaSuccess) {
      cudaGetLastError();
      return COSMA_ERR_NO_WORKSPACE;
    }
    cs.stage_bytes = want;
  }
  if (cap) cs.captured = true;
  uint8_t* wp = static_cast<uint8_t*>(cs.stage);
  R* Ar = reinterpret_cast<R*>(wp);
  R* Ai = reinterpret_cast<R*>(wp + a_b);
  R* Br = reinterpret_cast<R*>(wp + 2 * a_b);
  R* Bi = reinterpret_cast<R*>(wp + 2 * a_b + b_b);
  R* Tr = reinterpret_cast<R*>(wp + 2 * a_b + 2 * b_b);
  R* Ti = reinterpret_cast<R*>(wp + 2 * a_b + 2 * b_b + t_b);

  int rc = COSMA_OK;
  if (!no_ab) {
    split_complex_kernel<R><<<grid_for(a_rows * a_cols), 256, 0, st>>>(
        static_cast<const C2*>(A), a_rows, a_cols, lda, Ar, Ai, op_a == 2);
    count_launch();
    split_complex_kernel<R><<<grid_for(b_rows * b_cols), 256, 0, st>>>(
        static_cast<const C2*>(B), b_rows, b_cols, ldb, Br, Bi, op_b == 2);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return COSMA_ERR_CUDA;
    // Tr = Ar Br - Ai Bi,  Ti = Ar Bi + Ai Br
    const int64_t la = a_cols, lb = b_cols;
    rc = run_device_ex(m, n, k, Ar, la, Br, lb, Tr, n, engine, 1.0, 0.0, ta, tb, stream);
    if (rc == COSMA_OK)
      rc = run_device_ex(m, n, k, Ai, la, Bi, lb, Tr, n, engine, -1.0, 1.0, ta, tb, stream);
    if (rc == COSMA_OK)
      rc = run_device_ex(m, n, k, Ar, la, Bi, lb, Ti, n, engine, 1.0, 0.0, ta, tb, stream);
    if (rc == COSMA_OK)
      rc = run_device_ex(m, n, k, Ai, la, Br, lb, Ti, n, engine, 1.0, 1.0, ta, tb, stream);
    if (rc != COSMA_OK) return rc;
  } else {
    if (cudaMemsetAsync(Tr, 0, 2 * t_b, st) != cudaSuccess) return COSMA_ERR_CUDA;
  }
  combine_complex_kernel<R><<<grid_for(m * n), 256, 0, st>>>(
      m, n, Tr, Ti, static_cast<C2*>(C), ldc, alpha[0], alpha[1], beta[0], beta[1]);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? COSMA_OK : COSMA_ERR_CUDA;
}

}  // namespace
}  // namespace cosma

using namespace cosma;

extern "C" int cosma_zgemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k,
                           const double* alpha, const void* A, int64_t lda, const void* B,
                           int64_t ldb, const double* beta, void* C, int64_t ldc, int engine,
                           void* stream) {
  if (engine != COSMA_F64 && engine != COSMA_F64_EMU_BF16) return COSMA_ERR_UNSUPPORTED;
  return complex_gemm<double>(op_a, op_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, engine,
                              stream);
}

extern "C" int cosma_cgemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k,
                           const float* alpha, const void* A, int64_t lda, const void* B,
                           int64_t ldb, const float* beta, void* C, int64_t ldc, int engine,
                           void* stream) {
  if (engine != COSMA_F32 && engine != COSMA_F32_EMU_TF32) return COSMA_ERR_UNSUPPORTED;
  return complex_gemm<float>(op_a, op_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, engine,
                             stream);
}

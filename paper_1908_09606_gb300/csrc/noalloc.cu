// cosma_gemm_splitk_static: the split-k FP64/FP32 product with its partial
// sums in a fixed, statically allocated device array.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- code that records CUDA graphs in the global capture mode (where
// cudaMalloc is an illegal call), services that hand all device memory to
// their own pool at start-up and forbid allocations from libraries, and
// latency-critical loops that cannot afford the implicit synchronisation of
// cudaMalloc / cudaFree.  The regular entry points grow a library arena with
// cudaMalloc when a k split needs scratch; this one never does: it uses the
// array below, which every GPU that loads the library holds until the process
// exits.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress and caches it.  Make
// that first call before any stream capture.  Every call shares the one array
// and leaves its last contents behind; two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>
#include <mutex>

#include "internal.h"

namespace cosma {
namespace {

static __device__ __align__(256) unsigned char g_splitk_scratch[COSMA_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
void* g_static_addr[64] = {};

// Device address of g_splitk_scratch on the current device (looked up once).
int static_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return COSMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_splitk_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return COSMA_ERR_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return COSMA_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace cosma

using namespace cosma;

extern "C" int cosma_gemm_splitk_static(int64_t m, int64_t n, int64_t k, const void* A,
                                        int64_t lda, const void* B, int64_t ldb, void* C,
                                        int64_t ldc, int dtype, int pk, void* stream) {
  if (dtype != COSMA_F64 && dtype != COSMA_F32) return COSMA_ERR_UNSUPPORTED;
  if (m < 0 || n < 0 || k < 0 || pk < 1) return COSMA_ERR_INVALID_ARG;
  if (lda < (k > 1 ? k : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1))
    return COSMA_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return COSMA_OK;
  const int64_t w = dtype == COSMA_F64 ? 8 : 4;
  if (!C || (uintptr_t)C % w || !on_device(C)) return COSMA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (k == 0) {
    count_launch();
    return cudaMemset2DAsync(C, (size_t)(ldc * w), 0, (size_t)(n * w), (size_t)m, st) ==
                   cudaSuccess
               ? COSMA_OK
               : COSMA_ERR_CUDA;
  }
  if (!A || !B || (uintptr_t)A % w || (uintptr_t)B % w || !on_device(A) || !on_device(B))
    return COSMA_ERR_INVALID_ARG;
  // Scratch: pk partial m x n products (none when pk == 1).
  if (pk > 1 && (double)pk * (double)m * (double)n * (double)w > (double)COSMA_STATIC_SCRATCH_BYTES)
    return COSMA_ERR_NO_WORKSPACE;

  DeviceInfo info;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return COSMA_ERR_CUDA;
  info.device = dev;
  if (cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return COSMA_ERR_CUDA;
  cudaDeviceGetAttribute(&info.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&info.regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  // The active configuration (cosma_init), read without touching device state.
  // Planning is analytic: the learned selector runs its forward kernel on
  // buffers of its own, which this entry does not take.
  cosma_config cfg;
  if (cosma_get_config(&cfg) != COSMA_OK) return COSMA_ERR_INVALID_ARG;
  cosma_plan p;
  int rc = plan_gemm(m, n, k, dtype, COSMA_SELECT_ANALYTIC, info, cfg, &p, false);
  if (rc != COSMA_OK) return rc;
  // Balanced stripes over tiles x k slices.
  const int64_t tiles = ((m + p.tile_m - 1) / p.tile_m) * ((n + p.tile_n - 1) / p.tile_n);
  p.pk = pk;
  p.order = 1;
  p.pm = p.pn = 1;
  p.ctas = (int)(tiles * pk < info.sms ? tiles * pk : info.sms);
  rc = validate_plan(m, n, k, dtype, info, p);
  if (rc != COSMA_OK) return rc;

  void* scratch = nullptr;
  if (pk > 1) {
    rc = static_scratch(&scratch);
    if (rc != COSMA_OK) return rc;
  }
  const GemmArgs g{m, n, k, A, lda, B, ldb, C, ldc};
  const Sched sc = sched_from_plan(m, n, k, p);
  // Every (slice, row, column) partial the Reduce reads is written by exactly
  // one work unit first, so nothing in the array has to start at zero.
  int err = launch_simt(dtype, g, sc, scratch, nullptr, st);
  if (!err && pk > 1) err = launch_reduce(dtype, g, pk, scratch, st);
  return err == 0 ? COSMA_OK : COSMA_ERR_CUDA;
}

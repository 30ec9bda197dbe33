// Device half of the shared seeded input generator (Philox4x32-10, Salmon et
// al., SC'11).  The element-to-value mapping is the one stated in the package
// docstring of cosma_inputs; the host half (philox.py) implements the same
// published generator independently, and a GPU test checks the two agree bit
// for bit on sampled elements.  Nothing here belongs to the GEMM method.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// kind: 0 uniform, 1 integer, 2 loguniform.  Returns the f64 value; for the
// f32/bf16 uniform case the caller uses uniform_f32 instead.
__device__ __forceinline__ double value_f64(uint64_t e, int kind, uint64_t seed, uint32_t stream) {
  uint32_t c[4] = {(uint32_t)e, (uint32_t)(e >> 32), stream, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t w0 = c[0], w1 = c[1];
  if (kind == 0) {
    const uint64_t r53 = (w1 << 21) | (w0 >> 11);
    return ldexp((double)r53, -52) - 1.0;
  }
  if (kind == 1) return (double)((int)(w0 % 17u) - 8);
  const int e2 = (int)((w0 >> 1) % 54u) - 27;
  const double mant = 1.0 + ldexp((double)(w1 >> 9), -23);
  const double mag = ldexp(mant, e2);
  return (w0 & 1u) ? -mag : mag;
}

__device__ __forceinline__ float uniform_f32(uint64_t e, uint64_t seed, uint32_t stream) {
  uint32_t c[4] = {(uint32_t)e, (uint32_t)(e >> 32), stream, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t r24 = c[0] >> 8;
  return ldexpf((float)r24, -23) - 1.0f;  // exact: r24 < 2^24
}

template <typename T>
__global__ void fill_kernel(T* dst, int64_t rows, int64_t cols, int64_t ld, int kind,
                            uint64_t seed, uint32_t stream) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    T out;
    if constexpr (sizeof(T) == 8) {
      out = value_f64((uint64_t)e, kind, seed, stream);
    } else {
      const float f = (kind == 0) ? uniform_f32((uint64_t)e, seed, stream)
                                  : (float)value_f64((uint64_t)e, kind, seed, stream);
      if constexpr (sizeof(T) == 4) out = f;
      else out = __float2bfloat16_rn(f);
    }
    dst[r * ld + c] = out;
  }
}

}  // namespace

extern "C" {

// Fill a rows x cols matrix stored row-major with leading dimension ld
// (elements) at device pointer dst.  dtype: 0 f64, 1 f32, 2 bf16.
// kind: 0 uniform[-1,1), 1 integers in [-8,8], 2 loguniform.
// Returns 0 on success, a cudaError_t value otherwise.
int cosma_inputs_fill(void* dst, int64_t rows, int64_t cols, int64_t ld, int kind, int dtype,
                      uint64_t seed, uint32_t stream, void* cuda_stream) {
  if (rows < 0 || cols < 0 || ld < cols || kind < 0 || kind > 2 || dtype < 0 || dtype > 2)
    return (int)cudaErrorInvalidValue;
  if (rows == 0 || cols == 0) return 0;
  if (!dst) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t total = rows * cols;
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)sms * 16;
  if (blocks > cap) blocks = cap;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  switch (dtype) {
    case 0: fill_kernel<double><<<(unsigned)blocks, 256, 0, s>>>((double*)dst, rows, cols, ld, kind, seed, stream); break;
    case 1: fill_kernel<float><<<(unsigned)blocks, 256, 0, s>>>((float*)dst, rows, cols, ld, kind, seed, stream); break;
    default: fill_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>((__nv_bfloat16*)dst, rows, cols, ld, kind, seed, stream); break;
  }
  return (int)cudaGetLastError();
}

}  // extern "C"

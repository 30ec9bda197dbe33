// FP32 C-stationary tile with a multi-stage cp.async ring (K-F32 fast path).
//
// 128 x 128 C tile in registers (8 x 8 per thread: rows ty + 16 i, columns
// 4 tx + j and 64 + 4 tx + j), 16-deep k panels of A (row-major, pitch 20
// floats so the 16-byte fragment loads of a warp hit distinct banks) and B
// (row-major) streamed through STAGES shared-memory buffers by cp.async --
// the panels of round t + STAGES - 1 are in flight while round t is
// multiplied (the overlap of Sec. 7.3).  Ragged edges are zero-filled by the
// copy itself.  VEC = 4: 16-byte copies (A and B 16-byte aligned, lda and ldb
// multiples of 4); VEC = 1: 4-byte copies for any pitch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cosma {

constexpr int F32_BM = 128, F32_BN = 128, F32_BK = 16, F32_STAGES = 4;
constexpr int F32_APITCH = F32_BK + 4;

struct F32Smem {
  float As[F32_STAGES][F32_BM][F32_APITCH];
  float Bs[F32_STAGES][F32_BK][F32_BN];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int VEC>
__device__ __forceinline__ void f32_tile_async(const float* __restrict__ A, int64_t lda,
                                               const float* __restrict__ B, int64_t ldb,
                                               float* dst, int64_t ld, int64_t m, int64_t n,
                                               int64_t row0, int64_t col0, int64_t kbeg,
                                               int64_t kend, bool vec_out, F32Smem& sm) {
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int64_t nsteps = (kend - kbeg + F32_BK - 1) / F32_BK;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  auto issue = [&](int64_t step, int buf) {
    const int64_t k0 = kbeg + step * F32_BK;
    if constexpr (VEC == 4) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {  // A: 128 rows x 4 chunks of 4 floats
        const int idx = tid + e * 256;
        const int r = idx >> 2, c4 = idx & 3;
        const int64_t gr = row0 + r, gk = k0 + c4 * 4;
        int bytes = 0;
        const float* src = A;
        if (gr < m && gk < kend) {
          const int64_t left = kend - gk;
          bytes = left >= 4 ? 16 : (int)left * 4;
          src = A + gr * lda + gk;
        }
        cp_async16(&sm.As[buf][r][c4 * 4], src, bytes);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {  // B: 16 rows x 32 chunks of 4 floats
        const int idx = tid + e * 256;
        const int kr = idx >> 5, c4 = idx & 31;
        const int64_t gk = k0 + kr, gc = col0 + c4 * 4;
        int bytes = 0;
        const float* src = B;
        if (gk < kend && gc < n) {
          const int64_t left = n - gc;
          bytes = left >= 4 ? 16 : (int)left * 4;
          src = B + gk * ldb + gc;
        }
        cp_async16(&sm.Bs[buf][kr][c4 * 4], src, bytes);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {  // A: 128 rows x 16 floats
        const int idx = tid + e * 256;
        const int r = idx >> 4, c = idx & 15;
        const int64_t gr = row0 + r, gk = k0 + c;
        const bool in = gr < m && gk < kend;
        cp_async4(&sm.As[buf][r][c], in ? A + gr * lda + gk : A, in ? 4 : 0);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {  // B: 16 rows x 128 floats
        const int idx = tid + e * 256;
        const int kr = idx >> 7, c = idx & 127;
        const int64_t gk = k0 + kr, gc = col0 + c;
        const bool in = gk < kend && gc < n;
        cp_async4(&sm.Bs[buf][kr][c], in ? B + gk * ldb + gc : B, in ? 4 : 0);
      }
    }
  };

  __syncthreads();  // the previous tile's readers are done with the ring
#pragma unroll
  for (int s = 0; s < F32_STAGES - 1; ++s) {
    if (s < nsteps) issue(s, s);
    cp_async_commit();
  }
  for (int64_t st = 0; st < nsteps; ++st) {
    cp_async_wait<F32_STAGES - 2>();
    __syncthreads();
    {
      const int64_t nx = st + F32_STAGES - 1;
      if (nx < nsteps) issue(nx, (int)(nx % F32_STAGES));
      cp_async_commit();
    }
    const int buf = (int)(st % F32_STAGES);
#pragma unroll
    for (int kq = 0; kq < F32_BK; kq += 4) {
      float4 a4[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        a4[i] = *reinterpret_cast<const float4*>(&sm.As[buf][ty + 16 * i][kq]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kq + kk][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kq + kk][64 + tx * 4]);
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float a = kk == 0 ? a4[i].x : kk == 1 ? a4[i].y : kk == 2 ? a4[i].z : a4[i].w;
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a, b[j], acc[i][j]);
        }
      }
    }
  }
  cp_async_wait<0>();

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = row0 + ty + 16 * i;
    if (r >= m) continue;
    float* drow = dst + r * ld;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t c = col0 + h * 64 + tx * 4;
      if (vec_out && c + 4 <= n) {
        *reinterpret_cast<float4*>(drow + c) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < n) drow[c + j] = acc[i][4 * h + j];
      }
    }
  }
}

}  // namespace cosma

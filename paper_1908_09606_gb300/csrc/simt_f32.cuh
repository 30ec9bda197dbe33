// FP32 C-stationary tile on the FFMA pipe (K-F32).
//
// A BM x BN C tile stays in registers, 8 x (BN / 16) per thread.  Warps own
// 64 x (BN / 4) sub-tiles (BM = 128: 2 x 4 warps, 256 threads; BM = 256: 4 x 4
// warps, 512 threads, four warps per SM quarter to hide shared-memory latency).
// The 32 lanes of a warp form an 8 x 4 grid: lane (y, x) owns rows y, y + 8, ...,
// y + 56 of the warp tile and the column quads 4x + 16 g, g < BN / 64.
//
// Both panels keep their global layout in shared memory: A row-major with a
// 36-float pitch (k contiguous), so one 16-byte read gives a thread four k
// steps of one row and the 8 rows a warp reads at once fall in distinct bank
// quads; B row-major, two 16-byte reads per k step (4 distinct per warp).  Per
// 4 k steps a thread issues 8 + 8 shared loads for 256 FMAs, as 128 packed
// fma.rn.f32x2 (two round-to-nearest FMAs per issue slot: the results are those
// of scalar FMAs).  32-deep k panels
// stream through F32_STAGES buffers by cp.async (16-byte copies when A and B
// are 16-byte aligned with pitches a multiple of 4 floats, else 4-byte): the
// panels of round t + STAGES - 1 are in flight while round t is multiplied
// (the overlap of Sec. 7.3).  Ragged edges are zero-filled by the copies.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cosma {

constexpr int F32_BN = 128, F32_BK = 32, F32_STAGES = 4, F32_APITCH = F32_BK + 4;

template <int BM, int BN = F32_BN>
struct F32Smem {
  float As[F32_STAGES][BM][F32_APITCH];  // row-major A panel
  float Bs[F32_STAGES][F32_BK][BN];      // row-major B panel
};

// Threads of a CTA running f32_tile<BM>.
template <int BM>
__host__ __device__ constexpr int f32_threads() {
  return 2 * BM;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Two fp32 lanes in one 64-bit register pair, and the packed FMA on them
// (fma.rn.f32x2: two IEEE round-to-nearest FMAs, one issue slot).
__device__ __forceinline__ uint64_t f32x2_pack(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void f32x2_unpack(uint64_t v, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
__device__ __forceinline__ void f32x2_fma(uint64_t& d, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// C[row0 : row0 + BM, col0 : col0 + BN] (clipped to m x n) = A[rows, kbeg:kend] B[kbeg:kend, cols],
// written to dst (leading dimension ld).  Every thread of the CTA calls it.
template <int BM, int VEC, int BN = F32_BN>
__device__ __forceinline__ void f32_tile(const float* __restrict__ A, int64_t lda,
                                         const float* __restrict__ B, int64_t ldb, float* dst,
                                         int64_t ld, int64_t m, int64_t n, int64_t row0,
                                         int64_t col0, int64_t kbeg, int64_t kend, bool vec_out,
                                         F32Smem<BM, BN>& sm, float alpha = 1.f,
                                         float beta = 0.f) {
  static_assert(BN == 128 || BN == 256, "tile width");
  constexpr int NT = f32_threads<BM>();
  constexpr int NG = BN / 64;  // column quads per thread: 4x + 16 g
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int ar = (warp >> 2) * 64 + (lane >> 2);         // rows ar + 8 i, i = 0..7
  const int bc = (warp & 3) * (BN / 4) + (lane & 3) * 4;  // cols bc + 16 g .. + 3
  const int64_t nsteps = (kend - kbeg + F32_BK - 1) / F32_BK;

  // A copies: VEC-float chunks; this thread's chunk column a_c and rows
  // a_r + e * A_STEP.  A zero-fill copy reads nothing; its source is any valid
  // address.
  constexpr int A_COLS = F32_BK / VEC;       // chunks per A row
  constexpr int A_STEP = NT / A_COLS;        // A rows per pass of the CTA
  constexpr int A_PER = BM / A_STEP;
  const int a_r = tid / A_COLS, a_c = (tid % A_COLS) * VEC;
  const float* a_src = A + (kbeg + a_c);
  // B copies: a fixed chunk column per thread, rows b_k0 + e * B_STEP.
  constexpr int B_COLS = BN / VEC;
  constexpr int B_STEP = NT / B_COLS;
  constexpr int B_PER = F32_BK / B_STEP;
  const int b_k0 = tid / B_COLS, b_c = (tid % B_COLS) * VEC;
  const int64_t b_gc = col0 + b_c;
  const int b_bytes = b_gc >= n ? 0 : (n - b_gc >= VEC ? 4 * VEC : (int)(n - b_gc) * 4);
  const float* b_src = B + (b_bytes ? b_gc : 0) + (kbeg + b_k0) * ldb;

  // acc2[i][2 g + h] holds C(ar + 8 i, bc + 16 g + 2 h .. + 1): packed pairs for
  // fma.rn.f32x2
  uint64_t acc2[8][2 * NG];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 2 * NG; ++p) acc2[i][p] = f32x2_pack(0.f, 0.f);

  auto issue = [&](int64_t step, int buf) {
    const int64_t kk0 = step * F32_BK;  // offset from kbeg
    const int64_t kleft = kend - (kbeg + kk0 + a_c);
    const int a_bytes = kleft >= VEC ? 4 * VEC : (kleft > 0 ? (int)kleft * 4 : 0);
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int r = a_r + e * A_STEP;
      const int bytes = row0 + r < m ? a_bytes : 0;
      const float* src = bytes ? a_src + (row0 + r) * lda + kk0 : A;
      if constexpr (VEC == 4)
        cp_async16(&sm.As[buf][r][a_c], src, bytes);
      else
        cp_async4(&sm.As[buf][r][a_c], src, bytes);
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int kr = b_k0 + e * B_STEP;
      const int bytes = kbeg + kk0 + kr < kend ? b_bytes : 0;
      const float* src = bytes ? b_src + (kk0 + e * B_STEP) * ldb : B;
      if constexpr (VEC == 4)
        cp_async16(&sm.Bs[buf][kr][b_c], src, bytes);
      else
        cp_async4(&sm.Bs[buf][kr][b_c], src, bytes);
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
        a4[i] = *reinterpret_cast<const float4*>(&sm.As[buf][ar + 8 * i][kq]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint64_t b2[2 * NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const float4 u = *reinterpret_cast<const float4*>(&sm.Bs[buf][kq + kk][bc + 16 * g]);
          b2[2 * g] = f32x2_pack(u.x, u.y);
          b2[2 * g + 1] = f32x2_pack(u.z, u.w);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float a = kk == 0 ? a4[i].x : kk == 1 ? a4[i].y : kk == 2 ? a4[i].z : a4[i].w;
          const uint64_t a2 = f32x2_pack(a, a);
#pragma unroll
          for (int p = 0; p < 2 * NG; ++p) f32x2_fma(acc2[i][p], a2, b2[p]);
        }
      }
    }
  }
  cp_async_wait<0>();
  float acc[8][4 * NG];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 2 * NG; ++p) f32x2_unpack(acc2[i][p], acc[i][2 * p], acc[i][2 * p + 1]);

  // C = alpha acc + beta C (C read only when beta != 0)
  const bool plain = alpha == 1.f && beta == 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = row0 + ar + 8 * i;
    if (r >= m) continue;
    float* drow = dst + r * ld;
#pragma unroll
    for (int h = 0; h < NG; ++h) {
      const int64_t c = col0 + bc + 16 * h;
      if (!plain) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (c + j >= n) continue;
          float v = alpha * acc[i][4 * h + j];
          if (beta != 0.f) v = fmaf(beta, drow[c + j], v);
          drow[c + j] = v;
        }
      } else if (vec_out && c + 4 <= n) {
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

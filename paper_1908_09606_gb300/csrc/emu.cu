// Emulated FP64 GEMM on the bf16 tensor cores (K-SPLIT, K-EMU, K-RECOMB).
//
// Precision pattern (not in the paper; error-free splitting after Ozaki, Ogita,
// Oishi and Rump, Numer. Algorithms 59, 2012):
//
//  K-SPLIT  Row i of A is scaled by 2^-sigma_i (sigma_i: smallest power of two
//           above max_t |A_it|), column j of B by 2^-tau_j.  Each scaled
//           element becomes an integer F = round(|x| 2^(L - sigma)) (L = beta*s
//           - 1 bits, sign applied) taken straight from the FP64 bit pattern,
//           and F is written in s balanced base-2^beta digits d_1..d_s
//           (|d_q| <= 2^(beta-1)).  Digits are exact in bf16 (|d| <= 128).
//           No FP64 arithmetic is used.  Non-finite inputs set
//           COSMA_ERR_NONFINITE.
//  K-EMU    C_ij ~ 2^(sigma_i + tau_j - 2L) sum_{q,r} 2^(beta(2s - q - r)) (D^A_q D^B_r)_ij
//           over the truncated triangle q + r <= s + 1.  Pairs of one level
//           l = q + r share a scale, so a level is one product with an
//           extended k loop over its l-1 pairs.  Digit products are at most
//           2^(2 beta - 2), so an f32 tensor-memory accumulator is exact for
//           2^24 / 2^(2 beta - 2) products; the k loop is cut into groups of
//           that size and each group's exact integer sum is drained by the
//           epilogue warps into an exact float-float level sum kept in tensor
//           memory.  Two accumulators alternate so the MMAs of the next
//           group overlap the drain of this one.
//  K-RECOMB At the end of each level its exact sum is merged into a
//           float-float running total (high parts in shared memory, low parts
//           in registers: ten warps leave at most 168 registers a thread) (Horner, smallest
//           level first: T = T 2^-beta + L_l); after level 2 the tile is
//           converted to FP64 and scaled by 2^(sigma_i + tau_j + 2 - 2 beta).
//
// The C tile (128 x 128) is the paper's resident a x b tile (Listing 1); the
// slices of A and B stream through a 5-stage TMA ring exactly as in K-BF16.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cmath>
#include <mutex>

#include "tc_common.cuh"

namespace cosma {

namespace {

constexpr int EBM = 128, EBN = 128, EBK = 64, ESTAGES = 5;
constexpr int TPITCH = EBN + 1;  // padded row pitch of the running total in shared memory
constexpr int EMU_MAX_SLICES = 8;
constexpr int kExpNone = (int)0x80808080;  // memset(0x80) pattern: "no nonzero seen"

int emu_slices(const cosma_config& c) { return c.emu_slices > 0 ? c.emu_slices : 6; }
int emu_bits(const cosma_config& c) { return c.emu_slice_bits > 0 ? c.emu_slice_bits : 8; }

inline int64_t rup(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

// ---- K-SPLIT ----------------------------------------------------------------

// Exponent e with |x| < 2^e and |x| >= 2^(e-1); kExpNone for zero; flags
// non-finite values.
__device__ __forceinline__ int exp_above(double x, int* status) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & ((1ull << 52) - 1);
  if (E == 0x7FF) {
    atomicCAS(status, 0, (int)COSMA_ERR_NONFINITE);
    return kExpNone;
  }
  if (E == 0) {
    if (M == 0) return kExpNone;
    return -1074 + (64 - __clzll(M));
  }
  return E - 1022;
}

// Balanced digits of x relative to the scale exponent sigma (see file header).
__device__ __forceinline__ void split_digits(double x, int sigma, int L, int beta, int s,
                                             int (&d)[EMU_MAX_SLICES]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & ((1ull << 52) - 1);
  long long F = 0;
  if (E != 0x7FF && sigma != kExpNone && (E != 0 || M != 0)) {
    int e2;
    if (E == 0) e2 = -1074;
    else { M |= 1ull << 52; e2 = E - 1075; }
    const int sh = e2 + L - sigma;  // F = round(M 2^sh)
    if (sh >= 0) F = (long long)(M << sh);
    else {
      const int rs = -sh;
      if (rs <= 63) F = (long long)((M >> rs) + ((M >> (rs - 1)) & 1ull));
    }
    if (b >> 63) F = -F;
  }
  const long long base = 1LL << beta, half = base >> 1;
#pragma unroll
  for (int q = EMU_MAX_SLICES - 1; q >= 1; --q) {
    if (q < s) {
      long long r = F & (base - 1);
      if (r >= half) r -= base;
      d[q] = (int)r;
      F = (F - r) >> beta;
    } else {
      d[q] = 0;
    }
  }
  d[0] = (int)F;  // |F| <= 2^(beta-1) here
}

// sigma_i for every row of A (one block per row).
__global__ void row_exp_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda,
                               int* __restrict__ eA, int* status) {
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    int e = kExpNone;
    for (int64_t t = threadIdx.x; t < k; t += blockDim.x) e = max(e, exp_above(A[i * lda + t], status));
#pragma unroll
    for (int o = 16; o; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    __shared__ int red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
      int r = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = max(r, red[w]);
      eA[i] = r;
    }
    __syncthreads();
  }
}

// tau_j for every column of B: blocks of 256 columns x 256 rows, atomicMax.
__global__ void col_exp_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t ldb,
                               int* __restrict__ eB, int* status) {
  const int64_t j = blockIdx.x * 256 + threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.y * 256;
  if (j >= n) return;
  int e = kExpNone;
  const int64_t t1 = min(t0 + 256, k);
  for (int64_t t = t0; t < t1; ++t) e = max(e, exp_above(B[t * ldb + j], status));
  if (e != kExpNone) atomicMax(&eB[j], e);
}

// Slices of A: S[q][i][t] (ld kp), one thread per element.
__global__ void split_a_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda,
                               const int* __restrict__ eA, __nv_bfloat16* __restrict__ S,
                               int64_t kp, int s, int beta) {
  const int L = beta * s - 1;
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k, t = e - i * k;
    int d[EMU_MAX_SLICES];
    split_digits(A[i * lda + t], eA[i], L, beta, s, d);
#pragma unroll
    for (int q = 0; q < EMU_MAX_SLICES; ++q)
      if (q < s) S[((int64_t)q * m + i) * kp + t] = __float2bfloat16_rn((float)d[q]);
  }
}

// Slices of B, transposed to K-major: S[q][j][t] (ld kp).  32 x 32 tiles.
__global__ void split_b_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t ldb,
                               const int* __restrict__ eB, __nv_bfloat16* __restrict__ S,
                               int64_t kp, int s, int beta) {
  __shared__ __nv_bfloat16 tile[EMU_MAX_SLICES][32][34];
  const int L = beta * s - 1;
  const int64_t t0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t t = t0 + r, j = j0 + threadIdx.x;
    int d[EMU_MAX_SLICES];
    if (t < k && j < n) split_digits(B[t * ldb + j], eB[j], L, beta, s, d);
    else
#pragma unroll
      for (int q = 0; q < EMU_MAX_SLICES; ++q) d[q] = 0;
#pragma unroll
    for (int q = 0; q < EMU_MAX_SLICES; ++q)
      if (q < s) tile[q][threadIdx.x][r] = __float2bfloat16_rn((float)d[q]);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, t = t0 + threadIdx.x;
    if (j < n && t < k)
      for (int q = 0; q < s; ++q) S[((int64_t)q * n + j) * kp + t] = tile[q][r][threadIdx.x];
  }
}

// ---- K-EMU / K-RECOMB -------------------------------------------------------------

struct EmuArgs {
  Sched sch;           // tiles of 128 x 128, order 1, pk = 1
  int s, beta;
  int group_kb;        // k blocks of one pair per exact group at level 2 (2^(24-2beta+2)/64)
  const int* eA;
  const int* eB;
  double* C;
  int64_t ldc;
  int* status;
  long long wait_limit;
};

struct ELayout {
  static constexpr int A_BYTES = EBM * EBK * 2;
  static constexpr int B_BYTES = EBN * EBK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int T_OFF = ESTAGES * STAGE_BYTES;           // running total, high parts
  static constexpr int BAR_OFF = T_OFF + EBM * TPITCH * 4;
  static constexpr int NBARS = 2 * ESTAGES + 9;  // full, empty, tfull[4], tempty[4], drain
  static constexpr int TOTAL = BAR_OFF + NBARS * 8 + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x, int32_t y, int32_t z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// k blocks per pair in one exact group of a level with p pairs.
__device__ __forceinline__ int group_blocks(int group_kb, int p) {
  const int g = group_kb / p;
  return g > 0 ? g : 1;
}

// x * 2^e outside the exponent range of a normal double power of two.
__device__ __noinline__ double scale_slow(double x, int e) { return ldexp(x, e); }

__device__ __forceinline__ double scale_pow2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
  return scale_slow(x, e);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Epilogue warps (2..9) of K-EMU / K-RECOMB for the units of one CTA (or CTA
// pair): warp -> tensor-memory lane quadrant q4 = warp % 4 and column half h.
// Drains every exact group into the float-float level sum in tensor memory,
// merges finished levels into the running total (high parts in shared memory
// at Tsm, low parts in registers) and stores the FP64 tile.  Rows of this CTA
// start at tile_row * tile_rows + row_off.  tempty_addr: cluster addresses of
// the accumulator-free barriers of the MMA-issuing CTA.
template <bool IL>
__device__ __forceinline__ void emu_epilogue(const EmuArgs& a, int unit_cta, int64_t nunits,
                                             int64_t row_off, int64_t tile_rows,
                                             uint32_t tmem_base, uint8_t* Tsm,
                                             uint64_t* tfull, const uint32_t* tempty_addr,
                                             const tc::WaitCtx& w, int warp, int lane) {
  constexpr int NACC = IL ? 3 : 2;
  const int64_t kbt = a.sch.kbt;
  const int top = a.s + 1;
  const int q4 = warp & 3;
  const int h = (warp - 2) >> 2;
  const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
  const uint32_t col_lo = (uint32_t)(64 * h);
  const uint32_t lvl_hi_col = 256 + col_lo, lvl_lo_col = 384 + col_lo;
  const float down = 1.0f / (float)(1 << a.beta);
  float* Th = reinterpret_cast<float*>(Tsm) + (q4 * 32 + lane) * TPITCH + col_lo;
  uint32_t acc = 0;
  uint32_t tph[NACC];
#pragma unroll
  for (int b = 0; b < NACC; ++b) tph[b] = 0;
  bool ok = true;
  for (int64_t ui = 0; ui < nunits && ok; ++ui) {
    const Unit u = unit_of_cta(a.sch, unit_cta, ui);
    // Running total T = Th + Tl: Th in shared memory; Tl in registers (float-float
    // level sums) or, with int32 level sums, in tensor memory columns 384.. .
    float Tl[IL ? 1 : 64];
    int Lv[IL ? 64 : 1];  // exact level sum (int32 path)
    const uint32_t tl_col = 384 + col_lo;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      Th[j] = 0.f;
      if constexpr (!IL) Tl[j] = 0.f;
    }
    if constexpr (IL) {
      uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int c = 0; c < 64; c += 8) tc::tmem_st_32x8(tmem_base + lane_off + tl_col + c, z);
      tc::tmem_wait_st();
    }
    for (int lvl = top; lvl >= 2 && ok; --lvl) {
      const int p = lvl - 1;
      const int gk = group_blocks(a.group_kb, p);
      const int64_t ngroups = (kbt + gk - 1) / gk;
      for (int64_t g = 0; g < ngroups; ++g) {
        if (!tc::mbar_wait(&tfull[acc], tph[acc], w)) { ok = false; break; }
        tc::tc_fence_after();
        const bool first = (g == 0), last = (g == ngroups - 1);
        if constexpr (IL) {
          // Drain: the group's exact integer sums join the int32 level sum.
#pragma unroll
          for (int c = 0; c < 64; c += 8) {
            uint32_t v[8];
            tc::tmem_ld_32x8(tmem_base + lane_off + acc * EBN + col_lo + c, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int iv = __float2int_rn(__uint_as_float(v[j]));
              Lv[IL ? c + j : 0] = first ? iv : Lv[IL ? c + j : 0] + iv;
            }
          }
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive_remote(tempty_addr[acc]);
          tph[acc] ^= 1;
          acc = (acc + 1) % NACC;
          if (last) {
            // K-RECOMB: T = T * 2^-beta + level, the level split exactly into two floats.
#pragma unroll
            for (int c = 0; c < 64; c += 8) {
              uint32_t tl[8];
              tc::tmem_ld_32x8(tmem_base + lane_off + tl_col + c, tl);
              tc::tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int li = Lv[IL ? c + j : 0];
                const float lh = (float)li;
                const float ll = (float)(li - (int)lh);
                float s, e, nh, nl;
                two_sum(Th[c + j] * down, lh, s, e);
                e += __uint_as_float(tl[j]) * down + ll;
                fast_two_sum(s, e, nh, nl);
                Th[c + j] = nh;
                tl[j] = __float_as_uint(nl);
              }
              tc::tmem_st_32x8(tmem_base + lane_off + tl_col + c, tl);
            }
            tc::tmem_wait_st();
          }
        } else {
#pragma unroll
        for (int c = 0; c < 64; c += 8) {
          uint32_t v[8], hi[8], lo[8];
          tc::tmem_ld_32x8(tmem_base + lane_off + acc * EBN + col_lo + c, v);
          if (!first) {
            tc::tmem_ld_32x8(tmem_base + lane_off + lvl_hi_col + c, hi);
            tc::tmem_ld_32x8(tmem_base + lane_off + lvl_lo_col + c, lo);
          }
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float x = __uint_as_float(v[j]);  // exact integer
            float fh = x, fl = 0.f;
            if (!first) {
              float s, e;
              two_sum(__uint_as_float(hi[j]), x, s, e);
              fast_two_sum(s, __uint_as_float(lo[j]) + e, fh, fl);
            }
            if (last) {
              // K-RECOMB: T = T * 2^-beta + level (the first level processed starts T).
              float s, e, nh;
              two_sum(Th[c + j] * down, fh, s, e);
              e += Tl[IL ? 0 : c + j] * down + fl;
              fast_two_sum(s, e, nh, Tl[IL ? 0 : c + j]);
              Th[c + j] = nh;
            } else {
              hi[j] = __float_as_uint(fh);
              lo[j] = __float_as_uint(fl);
            }
          }
          if (!last) {
            tc::tmem_st_32x8(tmem_base + lane_off + lvl_hi_col + c, hi);
            tc::tmem_st_32x8(tmem_base + lane_off + lvl_lo_col + c, lo);
          }
        }
        tc::tmem_wait_st();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_remote(tempty_addr[acc]);
        tph[acc] ^= 1;
        acc = (acc + 1) % NACC;
        }
      }
    }
    if (!ok) break;
    // Final FP64 store of this thread's 64 columns of one row.
    const int64_t row = u.tile_row * tile_rows + row_off + q4 * 32 + lane;
    const int64_t cbase = u.tile_col * EBN + col_lo;
    const int ea = row < a.sch.m ? a.eA[row] : kExpNone;
    double* dst = a.C + row * a.ldc;
#pragma unroll
    for (int c = 0; c < 64; c += 8) {
      float tl[8];
      if constexpr (IL) {
        uint32_t t[8];
        tc::tmem_ld_32x8(tmem_base + lane_off + tl_col + c, t);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) tl[j] = __uint_as_float(t[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) tl[j] = Tl[IL ? 0 : c + j];
      }
      if (row < a.sch.m) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t col = cbase + c + j;
          if (col < a.sch.n) {
            const int eb = a.eB[col];
            const double val = (double)Th[c + j] + (double)tl[j];
            dst[col] = (ea == kExpNone || eb == kExpNone)
                           ? 0.0
                           : scale_pow2(val, ea + eb + 2 - 2 * a.beta);
          }
        }
      }
    }
  }
}

template <bool IL>
__global__ void __launch_bounds__(320, 1)
emu_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                EmuArgs a) {
  using L = ELayout;
  constexpr int NACC = IL ? 3 : 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + ESTAGES;
  uint64_t* tfull = empty + ESTAGES;
  uint64_t* tempty = tfull + 4;
  uint64_t* drain = tempty + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ESTAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NACC; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 8);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) tc::tmem_alloc(tslot, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const tc::WaitCtx w{a.wait_limit, a.status, abort_flag};
  const int cta = blockIdx.x;
  const int64_t nunits = units_of_cta(a.sch, cta);
  const int64_t kbt = a.sch.kbt;
  const int top = a.s + 1;

  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0, armed = 0, armed_ph = 0;
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        const Unit u = unit_of_cta(a.sch, cta, ui);
        bool ok = true;
        for (int lvl = top; lvl >= 2 && ok; --lvl) {
          const int p = lvl - 1;
          const int gk = group_blocks(a.group_kb, p);
          for (int64_t c0 = 0; c0 < kbt && ok; c0 += gk) {
            const int64_t c1 = min(c0 + gk, kbt);
            for (int q = 1; q <= p && ok; ++q) {
              for (int64_t kb = c0; kb < c1; ++kb) {
                if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) { ok = false; break; }
                tc::mbar_arrive_expect_tx(&full[stage], L::STAGE_BYTES);
                uint8_t* sa = smem + stage * L::STAGE_BYTES;
                tma_load_3d(sa, &tmA, &full[stage], (int32_t)(kb * EBK),
                            (int32_t)(u.tile_row * EBM), q - 1);
                tma_load_3d(sa + L::A_BYTES, &tmB, &full[stage], (int32_t)(kb * EBK),
                            (int32_t)(u.tile_col * EBN), lvl - q - 1);
                armed |= 1u << stage;
                armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
                if (++stage == ESTAGES) { stage = 0; ph ^= 1; }
              }
            }
          }
        }
        if (!ok) break;
      }
      if (*abort_flag) {
        for (int s = 0; s < ESTAGES; ++s) {
          if (!(armed >> s & 1)) continue;
          const long long t0 = clock64();
          while (!tc::mbar_try_wait(&full[s], (armed_ph >> s) & 1) &&
                 clock64() - t0 < tc::kDrainCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (tc::elect_one()) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(EBM, EBN);
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[NACC];
#pragma unroll
      for (int b = 0; b < NACC; ++b) aph[b] = 0;
      bool ok = true;
      for (int64_t ui = 0; ui < nunits && ok && !*abort_flag; ++ui) {
        for (int lvl = top; lvl >= 2 && ok; --lvl) {
          const int p = lvl - 1;
          const int gk = group_blocks(a.group_kb, p);
          for (int64_t c0 = 0; c0 < kbt && ok; c0 += gk) {
            const int64_t c1 = min(c0 + gk, kbt);
            if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t d = tmem_base + acc * EBN;
            bool first = true;
            for (int q = 1; q <= p && ok; ++q) {
              for (int64_t kb = c0; kb < c1; ++kb) {
                if (!tc::mbar_wait(&full[stage], ph, w)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
                const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < EBK / 16; ++kk) {
                  tc::mma_bf16(d, tc::smem_desc_sw128(sa + kk * 32),
                               tc::smem_desc_sw128(sb + kk * 32), idesc, first ? 0u : 1u);
                  first = false;
                }
                tc::mma_commit(&empty[stage]);
                if (++stage == ESTAGES) { stage = 0; ph ^= 1; }
              }
            }
            if (!ok) break;
            tc::mma_commit(&tfull[acc]);
            aph[acc] ^= 1;
            acc = (acc + 1) % NACC;
          }
        }
      }
      tc::mma_commit(drain);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  } else {
    uint32_t te[NACC];
#pragma unroll
    for (int b = 0; b < NACC; ++b) te[b] = tc::mapa_shared(&tempty[b], 0);
    emu_epilogue<IL>(a, cta, nunits, 0, EBM, tmem_base, smem + L::T_OFF, tfull, te, w, warp, lane);
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, 512);
  }
}


// ---- 2-SM variant ------------------------------------------------------------------
//
// A cluster of two CTAs computes a 256 x 128 tile with tcgen05.mma.cta_group::2
// (M = 256): each CTA loads its own 128 rows of the A slice and its own 64 of
// the 128 columns of the B slice (no multicast), the even CTA issues the MMAs
// and commits to the barriers of both, and each CTA drains its own 128 x 128
// accumulator exactly as the single-SM kernel does.  Per SM an MMA step then
// reads 6 KB of operands instead of 8 KB, and the ring is 6 stages deep.
constexpr int E2_STAGES = 6;

struct E2Layout {
  static constexpr int A_BYTES = EBM * EBK * 2;        // own 128 rows
  static constexpr int B_BYTES = (EBN / 2) * EBK * 2;  // own 64 columns
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int T_OFF = E2_STAGES * STAGE_BYTES;
  static constexpr int BAR_OFF = T_OFF + EBM * TPITCH * 4;
  static constexpr int NBARS = 2 * E2_STAGES + 9;
  static constexpr int TOTAL = BAR_OFF + NBARS * 8 + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};

__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int32_t x, int32_t y,
                                                 int32_t z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y), "r"(z)
      : "memory");
}

template <bool IL>
__global__ void __launch_bounds__(320, 1)
emu_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, EmuArgs a) {
  using L = E2Layout;
  constexpr int NACC = IL ? 3 : 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + E2_STAGES;
  uint64_t* tfull = empty + E2_STAGES;
  uint64_t* tempty = tfull + 4;
  uint64_t* drain = tempty + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = tc::cluster_ctarank();
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < E2_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);   // leader: its producer's arrival + both CTAs' bytes
      tc::mbar_init(&empty[s], 1);  // the leader's commit, multicast to both CTAs
    }
    for (int b = 0; b < NACC; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 16);  // leader: 8 epilogue warps of each CTA
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc_pair(tslot, 512);
  tc::tc_fence_before();
  tc::cluster_sync();  // barriers of both CTAs initialised, tensor memory allocated
  tc::tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const tc::WaitCtx w{a.wait_limit, a.status, abort_flag};
  const int pair = blockIdx.x >> 1;
  const int64_t nunits = units_of_cta(a.sch, pair);
  const int64_t kbt = a.sch.kbt;
  const int top = a.s + 1;

  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0;
      bool issued = false;
      uint32_t full_cl[E2_STAGES];
#pragma unroll
      for (int s = 0; s < E2_STAGES; ++s) full_cl[s] = tc::mapa_shared(&full[s], 0);
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        const Unit u = unit_of_cta(a.sch, pair, ui);
        bool ok = true;
        for (int lvl = top; lvl >= 2 && ok; --lvl) {
          const int p = lvl - 1;
          const int gk = group_blocks(a.group_kb, p);
          for (int64_t c0 = 0; c0 < kbt && ok; c0 += gk) {
            const int64_t c1 = min(c0 + gk, kbt);
            for (int q = 1; q <= p && ok; ++q) {
              for (int64_t kb = c0; kb < c1; ++kb) {
                if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) { ok = false; break; }
                if (leader) tc::mbar_arrive_expect_tx(&full[stage], 2 * L::STAGE_BYTES);
                uint8_t* sa = smem + stage * L::STAGE_BYTES;
                tma_load_3d_pair(sa, &tmA, full_cl[stage], (int32_t)(kb * EBK),
                                 (int32_t)(u.tile_row * (2 * EBM) + rank * EBM), q - 1);
                tma_load_3d_pair(sa + L::A_BYTES, &tmB, full_cl[stage], (int32_t)(kb * EBK),
                                 (int32_t)(u.tile_col * EBN + rank * (EBN / 2)), lvl - q - 1);
                issued = true;
                if (++stage == E2_STAGES) { stage = 0; ph ^= 1; }
              }
            }
          }
        }
        if (!ok) break;
      }
      if (*abort_flag && issued) {
        // Copies of this CTA signal the leader's barriers: give any still in
        // flight time to land before the pair leaves.
        const long long t0 = clock64();
        while (clock64() - t0 < (1LL << 22)) {
        }
      }
    }
  } else if (warp == 1) {
    if (leader && tc::elect_one()) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(2 * EBM, EBN);
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[NACC];
#pragma unroll
      for (int b = 0; b < NACC; ++b) aph[b] = 0;
      bool ok = true;
      for (int64_t ui = 0; ui < nunits && ok && !*abort_flag; ++ui) {
        for (int lvl = top; lvl >= 2 && ok; --lvl) {
          const int p = lvl - 1;
          const int gk = group_blocks(a.group_kb, p);
          for (int64_t c0 = 0; c0 < kbt && ok; c0 += gk) {
            const int64_t c1 = min(c0 + gk, kbt);
            if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t d = tmem_base + acc * EBN;
            bool first = true;
            for (int q = 1; q <= p && ok; ++q) {
              for (int64_t kb = c0; kb < c1; ++kb) {
                if (!tc::mbar_wait(&full[stage], ph, w)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
                const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < EBK / 16; ++kk) {
                  tc::mma_bf16_pair(d, tc::smem_desc_sw128(sa + kk * 32),
                                    tc::smem_desc_sw128(sb + kk * 32), idesc, first ? 0u : 1u);
                  first = false;
                }
                tc::mma_commit_pair(&empty[stage]);
                if (++stage == E2_STAGES) { stage = 0; ph ^= 1; }
              }
            }
            if (!ok) break;
            tc::mma_commit_pair(&tfull[acc]);
            aph[acc] ^= 1;
            acc = (acc + 1) % NACC;
          }
        }
      }
      tc::mma_commit_pair(drain);  // every MMA of the pair done (both CTAs' drain barriers)
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  } else {
    uint32_t te[NACC];
#pragma unroll
    for (int b = 0; b < NACC; ++b) te[b] = tc::mapa_shared(&tempty[b], 0);
    emu_epilogue<IL>(a, pair, nunits, (int64_t)rank * EBM, 2 * EBM, tmem_base, smem + L::T_OFF,
                     tfull, te, w, warp, lane);
  }
  __syncthreads();
  tc::tc_fence_before();
  tc::cluster_sync();  // no CTA leaves while its peer may still signal its barriers
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc_pair(tmem_base, 512);
}

int encode_tmap_slices(CUtensorMap* map, const void* base, int64_t rows, int64_t k, int64_t kp,
                       int s, int box_rows = EBM) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn) return COSMA_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)s};
  cuuint64_t strides[2] = {(cuuint64_t)(kp * 2), (cuuint64_t)(rows * kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)EBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

}  // namespace

long long emu_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_config& cfg) {
  const int s = emu_slices(cfg);
  const int64_t kp = rup(k, 8);
  return rup(m * 4, 256) + rup(n * 4, 256) + rup((int64_t)s * m * kp * 2, 256) +
         rup((int64_t)s * n * kp * 2, 256);
}

int launch_emu_bf16(const GemmArgs& g, const Sched& sch, const cosma_plan& p,
                    const cosma_config& cfg, void* ws, long long ws_bytes, int* status,
                    long long wait_limit, cudaStream_t st) {
  (void)p;
  const int s = emu_slices(cfg), beta = emu_bits(cfg);
  if (s < 2 || s > EMU_MAX_SLICES || beta < 2 || beta > 8 || beta * s - 1 > 62)
    return COSMA_ERR_INVALID_ARG;
  const bool pairs = sch.tile_m == 2 * EBM;
  if ((sch.tile_m != EBM && !pairs) || sch.tile_n != EBN || sch.k_block != EBK || sch.pk != 1)
    return COSMA_ERR_INVALID_ARG;
  const int64_t m = g.m, n = g.n, k = g.k, kp = rup(k, 8);
  if (emu_workspace_bytes(m, n, k, cfg) > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(g.A) & 7) || (reinterpret_cast<uintptr_t>(g.B) & 7) ||
      (reinterpret_cast<uintptr_t>(g.C) & 7))
    return COSMA_ERR_INVALID_ARG;
  uint8_t* w = static_cast<uint8_t*>(ws);
  int* eA = reinterpret_cast<int*>(w);
  w += rup(m * 4, 256);
  int* eB = reinterpret_cast<int*>(w);
  w += rup(n * 4, 256);
  __nv_bfloat16* SA = reinterpret_cast<__nv_bfloat16*>(w);
  w += rup((int64_t)s * m * kp * 2, 256);
  __nv_bfloat16* SB = reinterpret_cast<__nv_bfloat16*>(w);

  if (cudaMemsetAsync(eB, 0x80, (size_t)n * 4, st) != cudaSuccess) return (int)cudaGetLastError();
  const double* A = static_cast<const double*>(g.A);
  const double* B = static_cast<const double*>(g.B);
  {
    const int64_t blocks = m < 65535LL * 16 ? m : 65535LL * 16;
    row_exp_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, m, k, g.lda, eA, status);
    count_launch();
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)((k + 255) / 256));
    if (grid.y > 65535) return COSMA_ERR_UNSUPPORTED;
    col_exp_kernel<<<grid, 256, 0, st>>>(B, k, n, g.ldb, eB, status);
    count_launch();
  }
  {
    int64_t blocks = (m * k + 255) / 256;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    split_a_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, m, k, g.lda, eA, SA, kp, s, beta);
    count_launch();
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
    if (grid.y > 65535) return COSMA_ERR_UNSUPPORTED;
    split_b_kernel<<<grid, dim3(32, 8), 0, st>>>(B, k, n, g.ldb, eB, SB, kp, s, beta);
    count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;

  CUtensorMap ta, tb;
  int rc = encode_tmap_slices(&ta, SA, m, k, kp, s);
  if (rc != COSMA_OK) return rc;
  rc = encode_tmap_slices(&tb, SB, n, k, kp, s, pairs ? EBN / 2 : EBN);
  if (rc != COSMA_OK) return rc;

  EmuArgs args;
  args.sch = sch;
  args.s = s;
  args.beta = beta;
  // exact group: 2^24 / 2^(2 beta - 2) digit products, in 64-wide k blocks
  args.group_kb = (int)((1LL << (24 - 2 * beta + 2)) / EBK);
  if (args.group_kb < 1) args.group_kb = 1;
  args.eA = eA;
  args.eB = eB;
  args.C = static_cast<double*>(g.C);
  args.ldc = g.ldc;
  args.status = status;
  args.wait_limit = wait_limit;
  // Level sums fit in int32 when every level's products do: at most s pairs of
  // k products of magnitude <= 2^(2 beta - 2).
  const bool il = (double)s * (double)k * std::ldexp(1.0, 2 * beta - 2) < 2147483647.0;
  cudaError_t le;
  if (pairs) {
    void (*kern)(const CUtensorMap, const CUtensorMap, EmuArgs) =
        il ? emu_gemm_pair_kernel<true> : emu_gemm_pair_kernel<false>;
    const cudaError_t attr2 =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, E2Layout::ALLOC);
    if (attr2 != cudaSuccess) return (int)attr2;
    cudaLaunchConfig_t cfgl = {};
    cfgl.gridDim = dim3((unsigned)(2 * sch.ctas));
    cfgl.blockDim = dim3(320);
    cfgl.dynamicSmemBytes = E2Layout::ALLOC;
    cfgl.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfgl.attrs = at;
    cfgl.numAttrs = 1;
    prof_mark(st, true);
    le = cudaLaunchKernelEx(&cfgl, kern, ta, tb, args);
    prof_mark(st, false);
  } else {
    void (*kern)(const CUtensorMap, const CUtensorMap, EmuArgs) =
        il ? emu_gemm_kernel<true> : emu_gemm_kernel<false>;
    const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, ELayout::ALLOC);
    if (attr != cudaSuccess) return (int)attr;
    prof_mark(st, true);
    kern<<<sch.ctas, 320, ELayout::ALLOC, st>>>(ta, tb, args);
    prof_mark(st, false);
    le = cudaGetLastError();
  }
  if (le != cudaSuccess) return (int)le;
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace cosma

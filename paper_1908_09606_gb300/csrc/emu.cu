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
//           l = q + r share a scale.  Digit products are at most 2^(2 beta - 2),
//           so an f32 tensor-memory accumulator is exact for 2^24 / 2^(2 beta - 2)
//           products; the k loop is cut into groups of that size, and each
//           group's exact integer sum is drained by the epilogue warps into an
//           int32 level sum held in registers.  k is walked in super-chunks of
//           4096 (all levels per chunk), so a level sum stays below 2^31 for any
//           k.  Two (256-wide tiles) or four (128-wide tiles) accumulator
//           buffers let the MMAs of the next groups overlap a drain.
//  K-RECOMB Within a chunk, levels are taken in pairs: the lower level's sum
//           keeps its low beta bits as digits and carries the rest into the
//           next level's sum, and at the end of each pair the exact value
//           L_l + 2^beta L_(l-1) joins an exact int64 fixed-point running total
//           kept in global scratch (L2 reductions; see "Running total" below);
//           after the last chunk the tile is converted to FP64 once, so every
//           kernel and tile shape gives the same bits: the method's exact result
//           rounded once (level pairs below the fixed-point base aside).
//
// The C tile (128 x 128 on one SM, or 256 x 256 / 256 x 128 on a CTA pair with
// tcgen05.mma.cta_group::2) is the resident a x b block of C of the paper's
// sequential schedule (Sec. 5.2); the slices of A and B stream through a TMA
// ring (7 stages of 32 KB, 9 of 24 KB for 256 x 128 pairs).  Pairs launched
// cooperatively advance in lock-step super-chunks (bounded waits) so that
// concurrent tiles read the same slice panels from L2.
//
// k split (the parallel schedule's pk > 1, Sec. 6.1, for products with few C
// tiles): k is cut at super-chunk boundaries, each unit (tile, k slice) ends
// with its exact fixed-point total, and the units' totals are summed exactly in
// an int64 array (L2 reductions) that a finishing pass rounds to FP64 -- the
// integers an unsplit product sums, so the split changes no bit of C.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "tc_common.cuh"

namespace cosma {

namespace {

constexpr int EBM = 128, EBN = 128, EBK = 64, ESTAGES = 7;
// Slice layout, k-blocked (the paper's blocked data layout, Sec. 7.6): slice q of
// an operand with R rows is stored as ceil(k / EKB) panels of R x EKB, element
// (i, t) at ((q nkb + t / EKB) R + i) EKB + t % EKB, zero beyond k.  A TMA box
// (64 k by 128 rows) then spans 128 rows of 4 KB -- a few pages -- however long
// k is (row-major slices with k = 2^20 put every row of a box in its own page).
constexpr int64_t EKB = 2048;
constexpr int EMU_MAX_SLICES = 8;
constexpr int kExpNone = (int)0x80808080;  // memset(0x80) pattern: "no nonzero seen"

int emu_slices(const cosma_config& c) { return c.emu_slices > 0 ? c.emu_slices : 6; }
int emu_bits(const cosma_config& c) { return c.emu_slice_bits > 0 ? c.emu_slice_bits : 8; }

inline int64_t rup(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

// k rounded up to whole layout panels.
inline int64_t emu_kpad(int64_t k) { return rup(k > 0 ? k : 1, EKB); }

__device__ __forceinline__ int64_t slice_at(int q, int64_t i, int64_t t, int64_t rows,
                                            int64_t nkb) {
  return (((int64_t)q * nkb + t / EKB) * rows + i) * EKB + (t % EKB);
}

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

// F = round(|x| 2^(L - sigma)) with the sign of x, from the FP64 bit pattern
// (0 for zero, non-finite x or an all-zero row / column).
__device__ __forceinline__ long long scaled_integer(double x, int sigma, int L) {
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
  return F;
}

// Balanced digits of x relative to the scale exponent sigma (see file header).
__device__ __forceinline__ void split_digits(double x, int sigma, int L, int beta, int s,
                                             int (&d)[EMU_MAX_SLICES]) {
  long long F = scaled_integer(x, sigma, L);
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

// The same digits for the default 6 slices of 8 bits (L = 47) in 32-bit
// arithmetic: with F = hi 2^24 + lo, 0 <= lo < 2^24, the three low digits come
// from lo alone, their carry (0 or 1) joins hi, and hi gives the rest.
__device__ __forceinline__ void split_digits_6x8(double x, int sigma, int (&d)[EMU_MAX_SLICES]) {
  const long long F = scaled_integer(x, sigma, 47);
  int lo = (int)(F & 0xFFFFFF);
  int hi = (int)(F >> 24);
#pragma unroll
  for (int q = 5; q >= 3; --q) {
    int r = lo & 255;
    if (r >= 128) r -= 256;
    d[q] = r;
    lo = (lo - r) >> 8;
  }
  hi += lo;
#pragma unroll
  for (int q = 2; q >= 1; --q) {
    int r = hi & 255;
    if (r >= 128) r -= 256;
    d[q] = r;
    hi = (hi - r) >> 8;
  }
  d[0] = hi;
#pragma unroll
  for (int q = 6; q < EMU_MAX_SLICES; ++q) d[q] = 0;
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

// Slices of A in the k-blocked layout (slice_rows rows per panel), zeros for
// k <= t < kpad.  Each thread takes 4 consecutive t of a row (x: columns in
// groups of 4, y: rows in steps of gridDim.y) and writes 8 bytes per slice.
__global__ void split_a_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda,
                               const int* __restrict__ eA, __nv_bfloat16* __restrict__ S,
                               int64_t kpad, int64_t slice_rows, int s, int beta) {
  const int L = beta * s - 1;
  const int64_t nkb = kpad / EKB;
  const int64_t t0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (t0 >= kpad) return;
  const bool fast = s == 6 && beta == 8;
  for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
    const int sigma = eA[i];
    const double* row = A + i * lda;
    int d[4][EMU_MAX_SLICES];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t t = t0 + v;
      const double x = t < k ? row[t] : 0.0;
      if (fast) split_digits_6x8(x, sigma, d[v]);
      else split_digits(x, sigma, L, beta, s, d[v]);
    }
#pragma unroll
    for (int q = 0; q < EMU_MAX_SLICES; ++q) {
      if (q >= s) break;
      __nv_bfloat162 lo2, hi2;
      lo2.x = __float2bfloat16_rn((float)d[0][q]);
      lo2.y = __float2bfloat16_rn((float)d[1][q]);
      hi2.x = __float2bfloat16_rn((float)d[2][q]);
      hi2.y = __float2bfloat16_rn((float)d[3][q]);
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&lo2);
      pk.y = *reinterpret_cast<uint32_t*>(&hi2);
      *reinterpret_cast<uint2*>(S + slice_at(q, i, t0, slice_rows, nkb)) = pk;
    }
  }
}

// Slices of B, transposed to K-major, in the k-blocked layout (zeros for
// k <= t < kpad).  32 x 32 tiles through shared memory (row pitch 36: 8-byte
// aligned rows); each thread then writes 4 consecutive t of one column j per
// slice as one 8-byte store.  The grid covers kpad.
__global__ void split_b_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t ldb,
                               const int* __restrict__ eB, __nv_bfloat16* __restrict__ S,
                               int64_t kpad, int64_t slice_rows, int s, int beta) {
  __shared__ __align__(8) __nv_bfloat16 tile[EMU_MAX_SLICES][32][36];
  const int L = beta * s - 1;
  const int64_t nkb = kpad / EKB;
  const int64_t t0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const bool fast = s == 6 && beta == 8;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t t = t0 + r, j = j0 + threadIdx.x;
    int d[EMU_MAX_SLICES];
    if (t < k && j < n) {
      if (fast) split_digits_6x8(B[t * ldb + j], eB[j], d);
      else split_digits(B[t * ldb + j], eB[j], L, beta, s, d);
    } else {
#pragma unroll
      for (int q = 0; q < EMU_MAX_SLICES; ++q) d[q] = 0;
    }
#pragma unroll
    for (int q = 0; q < EMU_MAX_SLICES; ++q)
      if (q < s) tile[q][threadIdx.x][r] = __float2bfloat16_rn((float)d[q]);
  }
  __syncthreads();
  const int lid = threadIdx.y * 32 + threadIdx.x;  // 0..255: column jj, 4-group g
  const int jj = lid >> 3, g = lid & 7;
  const int64_t j = j0 + jj, t = t0 + 4 * g;
  if (j < n && t < kpad) {
    for (int q = 0; q < s; ++q)
      *reinterpret_cast<uint2*>(S + slice_at(q, j, t, slice_rows, nkb)) =
          *reinterpret_cast<const uint2*>(&tile[q][jj][4 * g]);
  }
}

// ---- K-EMU / K-RECOMB -------------------------------------------------------------
//
// Iteration order of one unit (a C tile over the k blocks [kb0, kb1) of its k
// slice; all roles walk it identically):
//   for each k super-chunk [sc0, sc1) of kcb k-blocks in [kb0, kb1)
//     for each level l = s+1 down to 2 (p = l - 1 slice pairs)
//       for each exact group [c0, c1) of gk(p) k-blocks inside the super-chunk
//         for each pair q = 1..p:  for each k-block kb in [c0, c1):
//           D[acc] (+)= A_q[tile rows, kb] * B_{l-q}[tile cols, kb]
//       (the group's f32 sums are exact integers: drained into an int32 level sum)
//     (end of every second level in the super-chunk: the exact value of the level
//      pair joins the fixed-point running total, see the epilogue)
// Each level re-reads the super-chunk's slice panels; shorter super-chunks keep
// them in L2 across the levels at the price of more merges of the running total.

struct EmuArgs {
  Sched sch;           // tiles (128 x 128, or 256 x 256 / 256 x 128 pairs), order 1; units
                       // from emu_unit_of_cta (k slices of whole super-chunks)
  int s, beta;
  int group_kb;        // k blocks of one pair per exact group (2^(24 - 2 beta + 2) / 64)
  int chunk_kb;        // k blocks per super-chunk
  const int* eA;
  const int* eB;
  double* C;
  int64_t ldc;
  int* status;
  long long wait_limit;
  unsigned int* lockstep;  // cooperative launches: per-unit progress counter (zeroed), else null
  long long* T;            // per-CTA running totals, 128 x tile_n int64 each
  int t_base;              // fixed-point base of T (see "Running total")
  double alpha, beta_c;    // C = alpha A B + beta_c C (C read only when beta_c != 0)
  long long* X;            // pk > 1: the units' totals are summed here ([m][n], zeroed),
                           // and emu_finish_kernel forms C; null: units write C
};

// One 64 (k) x rows box of slice q at k-block kb and row y of the k-blocked layout.
__device__ __forceinline__ void tma_load_slice(void* dst, const CUtensorMap* map, uint64_t* bar,
                                               int64_t kb, int32_t y, int32_t q) {
  const int64_t t = kb * EBK;
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];\n" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_u32(bar)), "r"((int32_t)(t % EKB)),
      "r"(y), "r"((int32_t)(t / EKB)), "r"(q)
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

// Running total (both kernels).  Tensor memory holds only accumulators (512 /
// BN buffers of BN columns).  The exact level sum of the current super-chunk
// stays in registers (BN / 2 int32 per epilogue thread, and BN / 8 words of
// digits while a level pair is open), and the running total of the tile is an
// exact int64 fixed-point number
// T = sum_chunks sum_l 2^(beta (s + 1 - l) - base) L_l kept
// in a per-CTA scratch region in global memory: the first merge of a tile
// stores, later ones are reductions performed in L2, and the thread that made
// them reads the total back (L2 only) and forms the FP64 result,
// C = T 2^(sigma_i + tau_j + 2 - beta (s + 1) + base).  (Adding the unit's last
// level sum in registers at the read-back instead of merging it cost 12 % on
// 65536 x 65536 x 1024 -- one super-chunk per tile -- on one GB300; square
// 16384^3 moved by less than the run-to-run spread.)  `base` (host, from k)
// keeps |T| < 2^62; a level pair whose weight is below 2^base is rounded to it
// (one rounding per pair and super-chunk).

// v 2^sh as an int64 (sh < 0: rounded to nearest, ties up).
__device__ __forceinline__ long long fx_shift(long long v, int sh) {
  if (sh >= 0) return v << sh;
  return (v + (1LL << (-sh - 1))) >> (-sh);
}

// 8 x 8 transpose within each group of 8 lanes: on entry lane l holds row l of
// the group's block (v[j] = entry (l % 8, j)), on return column l % 8 (v[i] =
// entry (i, l % 8)).  Three butterfly stages: at stage sb, entries whose row and
// column differ in bit sb trade places with lane ^ sb.
template <class V>
__device__ __forceinline__ void transpose8(V (&v)[8], int l8) {
#pragma unroll
  for (int sb = 4; sb >= 1; sb >>= 1) {
#pragma unroll
    for (int i0 = 0; i0 < 8; ++i0) {
      if (i0 & sb) continue;
      const bool up = (l8 & sb) != 0;
      const V send = up ? v[i0] : v[i0 | sb];
      const V recv = __shfl_xor_sync(0xffffffffu, send, sb);
      if (up) v[i0] = recv;
      else v[i0 | sb] = recv;
    }
  }
}

// Epilogue warps W0 .. W0 + 7 of K-EMU / K-RECOMB for the units of one CTA (or
// CTA pair): warp -> tensor-memory lane quadrant q4 = warp % 4 and column half
// h; each thread owns one row and BN / 2 columns of this CTA's 128 rows, which
// start at row tile_row * TM + row_off.  Its entries of the running total sit
// at Tt + c * 128 (c = its column), so a warp touches 32 consecutive int64 per
// column.  tempty_addr: cluster addresses of the accumulator-free barriers of
// the MMA-issuing CTA.
template <int BN, int TM, int W0>
__device__ __forceinline__ void emu_fx_epilogue(const EmuArgs& a, int unit_cta, int64_t nunits,
                                                int64_t row_off, uint32_t tmem_base,
                                                uint64_t* tfull, const uint32_t* tempty_addr,
                                                const tc::WaitCtx& w, int warp, int lane) {
  constexpr int HC = BN / 2;
  constexpr int NACC = 512 / BN;
  const int top = a.s + 1;
  const int q4 = warp & 3;
  const int h = (warp - W0) >> 2;
  const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
  const uint32_t col_lo = (uint32_t)(HC * h);
  long long* Tt = a.T + (int64_t)blockIdx.x * (128 * BN) + ((int64_t)h * HC * 4 + q4) * 32 + lane;
  // The running totals (about 39 MB for all CTAs) stay in L2 between merges
  // while the slice panels stream past them: their lines are the last to go.
  uint64_t keep;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
  uint32_t acc = 0;
  uint32_t tph[NACC];
#pragma unroll
  for (int b = 0; b < NACC; ++b) tph[b] = 0;
  const int l8 = lane & 7, g8 = lane >> 3;
  const int eoff = 2 - a.beta * top + a.t_base;
  // the read-back addresses from an opaque copy of the base, so the compiler does
  // not keep the merges' per-column addresses live across the loops
  long long* Tf = Tt;
  asm volatile("" : "+l"(Tf));

  // Deferred FP64 store.  A finished unit's total is read back and stored in NB
  // batches of 8 columns, two after each group drain of the next unit's first
  // level (the accumulator is already free, so the MMAs run on meanwhile), and any
  // left at the end of that level, before the unit's first merge overwrites the
  // total; after the last unit, all at once.  Same thread, same addresses: each
  // load precedes the next unit's store in program order, so it reads the
  // finished total.
  constexpr int NB = HC / 8;
  int pb = NB;  // next batch of the pending unit (NB: nothing pending)
  int64_t p_row0 = 0, p_cbase = 0;
  int p_ea = kExpNone;
  // batches pb .. lim - 1 (lim - pb even), two at a time with both loads in flight:
  // C = T 2^(sigma_i + tau_j + 2 - beta (s + 1) + base) for the thread's row, 8
  // columns each, formed in the row's lane, transposed within groups of 8 lanes and
  // written as four 64-byte row segments per instruction
  auto rb_upto = [&](int lim) {
#pragma unroll 1
    for (; pb < lim; pb += 2) {
      long long tv[2][8];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          asm volatile("ld.relaxed.gpu.global.L2::cache_hint.s64 %0, [%1], %2;"
                       : "=l"(tv[b][j])
                       : "l"(Tf + (8 * (pb + b) + j) * 128), "l"(keep)
                       : "memory");
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int c = 8 * (pb + b);
        const int64_t col = p_cbase + c + l8;
        int eb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          eb[j] = p_cbase + c + j < a.sch.n ? a.eB[p_cbase + c + j] : kExpNone;
        double v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          double x = (p_ea == kExpNone || eb[j] == kExpNone)
                         ? 0.0
                         : scale_pow2((double)tv[b][j], p_ea + eb[j] + eoff);
          if (a.alpha != 1.0) x *= a.alpha;
          v[j] = x;
        }
        transpose8(v, l8);
        // now v[i] = C(p_row0 + 8 g8 + i, p_cbase + c + l8)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int64_t r = p_row0 + 8 * g8 + i;
          if (r < a.sch.m && col < a.sch.n) {
            double* dst = a.C + r * a.ldc + col;
            double x = v[i];
            if (a.beta_c != 0.0) x = fma(a.beta_c, *dst, x);
            *dst = x;
          }
        }
      }
    }
  };

  bool ok = true;
  const int dmask = (1 << a.beta) - 1;
  for (int64_t ui = 0; ui < nunits && ok; ++ui) {
    const Unit u = emu_unit_of_cta(a.sch, unit_cta, ui);
    int Lv[HC];           // exact level sum of the current super-chunk
    uint32_t dg[HC / 4];  // low digits of a pair's lower level, four 8-bit fields a word
    bool stored = false;
    for (int64_t sc0 = u.kb0; sc0 < u.kb1 && ok; sc0 += a.chunk_kb) {
      const int64_t sc1 = min(sc0 + (int64_t)a.chunk_kb, u.kb1);
      // one exact group: its integer sums join Lv (the level's first group sets it,
      // unless Lv starts from a carry)
      auto drain = [&](auto first_tag) -> bool {
        constexpr bool kFirst = decltype(first_tag)::value;
        if (!tc::mbar_wait(&tfull[acc], tph[acc], w)) return false;
        tc::tc_fence_after();
        const uint32_t src = tmem_base + lane_off + acc * BN + col_lo;
#pragma unroll
        for (int c = 0; c < HC; c += 16) {
          uint32_t v[16];
          tc::tmem_ld_32x16(src + c, v);
          tc::tmem_wait_ld_r16(v);  // the registers are read only after the wait
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int iv = __float2int_rn(__uint_as_float(v[j]));  // exact integer
            Lv[c + j] = kFirst ? iv : Lv[c + j] + iv;
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_remote_relaxed(tempty_addr[acc]);
        tph[acc] ^= 1;
        acc = (acc + 1) == NACC ? 0 : acc + 1;
        return true;
      };
      // Levels join the running total two at a time (K-RECOMB).  The lower level
      // lvl of a pair keeps its low beta bits as digits and passes the rest,
      // floor(L_lvl / 2^beta), on as the start of level lvl - 1's sum, which then
      // ends at L_{lvl-1} + floor(L_lvl / 2^beta) (one super-chunk's level sums
      // stay below 2^29.6, so this fits an int32); the pair's value is
      // 2^beta (that sum) + digits = L_lvl + 2^beta L_{lvl-1}, exactly, and
      // T += value 2^(beta (top - lvl) - base).  With an odd number of levels the
      // last, lvl = 2, joins alone.
      for (int lvl = top; lvl >= 2 && ok; lvl -= 2) {
        const bool pair = lvl > 2;
        if (pair) {
          const int gk = group_blocks(a.group_kb, lvl - 1);
          for (int64_t c0 = sc0; c0 < sc1; c0 += gk) {
            if (!(c0 == sc0 ? drain(std::true_type{}) : drain(std::false_type{}))) {
              ok = false;
              break;
            }
            // the previous unit's store: two batches per group, the rest at the
            // end of this (its first) level
            if (pb < NB) rb_upto(c0 + gk >= sc1 ? NB : min(NB, pb + 2));
          }
          if (!ok) break;
#pragma unroll
          for (int c = 0; c < HC; c += 4) {
            uint32_t wd = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              wd |= (uint32_t)(Lv[c + j] & dmask) << (8 * j);
              Lv[c + j] >>= a.beta;  // floor: L = 2^beta (L >> beta) + (L & mask)
            }
            dg[c / 4] = wd;
          }
        }
        {
          const int hl = pair ? lvl - 1 : lvl;
          const int gk = group_blocks(a.group_kb, hl - 1);
          for (int64_t c0 = sc0; c0 < sc1; c0 += gk) {
            if (!(c0 == sc0 && !pair ? drain(std::true_type{}) : drain(std::false_type{}))) {
              ok = false;
              break;
            }
          }
          if (!ok) break;
        }
        const int sh = a.beta * (top - lvl) - a.t_base;
        // (8 columns at a time: each batch's shifted values are sent before the next
        // is formed, which keeps the 64-bit temporaries few)
#pragma unroll
        for (int c = 0; c < HC; c += 8) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long long lv =
                pair ? ((long long)Lv[c + j] << a.beta) +
                           (long long)((dg[(c + j) / 4] >> (8 * ((c + j) % 4))) & 0xFFu)
                     : (long long)Lv[c + j];
            const long long x = fx_shift(lv, sh);
            // relaxed gpu-scope store, reductions and read-back: same-address
            // operations of one thread stay in program order (coherence)
            if (!stored)
              asm volatile("st.relaxed.gpu.global.L2::cache_hint.s64 [%0], %1, %2;" ::"l"(
                               Tt + (c + j) * 128),
                           "l"(x), "l"(keep)
                           : "memory");
            else
              asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(
                               Tt + (c + j) * 128),
                           "l"(x), "l"(keep)
                           : "memory");
          }
        }
        stored = true;
      }
    }
    if (!ok) break;
    const int64_t row0 = u.tile_row * TM + row_off + q4 * 32;
    const int64_t cbase = u.tile_col * BN + col_lo;
    if (a.X) {
      // k split: the unit's exact total joins the product's,
      // transposed like the FP64 store, by L2 reductions -- integer sums, so
      // the order of the k slices changes nothing
#pragma unroll 1
      for (int c = 0; c < HC; c += 8) {
        long long tv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          asm volatile("ld.relaxed.gpu.global.L2::cache_hint.s64 %0, [%1], %2;"
                       : "=l"(tv[j])
                       : "l"(Tt + (c + j) * 128), "l"(keep)
                       : "memory");
        transpose8(tv, l8);
        const int64_t col = cbase + c + l8;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int64_t r = row0 + 8 * g8 + i;
          if (r < a.sch.m && col < a.sch.n)
            asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(a.X + r * a.sch.n + col),
                         "l"(tv[i])
                         : "memory");
        }
      }
      continue;
    }
    // this unit's FP64 store waits for the next unit's first level, which is
    // always the lower level of a pair (the host takes s >= 2 slices)
    p_row0 = row0;
    p_cbase = cbase;
    p_ea = row0 + lane < a.sch.m ? a.eA[row0 + lane] : kExpNone;
    pb = 0;
  }
  if (ok && pb < NB) rb_upto(NB);
}

// Same iteration order for the producer and the MMA issuer over the k blocks
// [kb0, kb1) of a unit: calls body(q, lvl, kb) for every k-block of every pair,
// and group_begin / group_end around the exact groups.  Returns false as soon as
// a callback does (abort).  chunk_begin(c) runs before super-chunk c (0, 1, ...)
// of the unit.
template <class ChunkBegin, class GroupBegin, class Body, class GroupEnd>
__device__ __forceinline__ bool emu_walk_chunks(const EmuArgs& a, int64_t kb0, int64_t kb1,
                                                ChunkBegin chunk_begin, GroupBegin group_begin,
                                                Body body, GroupEnd group_end) {
  const int top = a.s + 1;
  int64_t chunk = 0;
  for (int64_t sc0 = kb0; sc0 < kb1; sc0 += a.chunk_kb, ++chunk) {
    if (!chunk_begin(chunk)) return false;
    const int64_t sc1 = min(sc0 + (int64_t)a.chunk_kb, kb1);
    for (int lvl = top; lvl >= 2; --lvl) {
      const int p = lvl - 1;
      const int gk = group_blocks(a.group_kb, p);
      for (int64_t c0 = sc0; c0 < sc1; c0 += gk) {
        const int64_t c1 = min(c0 + (int64_t)gk, sc1);
        if (!group_begin()) return false;
        bool first = true;
        for (int q = 1; q <= p; ++q)
          for (int64_t kb = c0; kb < c1; ++kb) {
            if (!body(q, lvl, kb, first)) return false;
            first = false;
          }
        group_end();
      }
    }
  }
  return true;
}

template <class GroupBegin, class Body, class GroupEnd>
__device__ __forceinline__ bool emu_walk(const EmuArgs& a, int64_t kb0, int64_t kb1,
                                         GroupBegin group_begin, Body body, GroupEnd group_end) {
  return emu_walk_chunks(a, kb0, kb1, [](int64_t) { return true; }, group_begin, body, group_end);
}

// k-block range of unit i of CTA (or pair) `cta` alone, for the MMA issuer.
__device__ __forceinline__ void emu_unit_range(const Sched& s, int cta, int64_t i, int64_t& kb0,
                                               int64_t& kb1) {
  if (s.pk == 1) {
    kb0 = 0;
    kb1 = s.kbt;
    return;
  }
  const int64_t unit = cta + i * (int64_t)s.ctas;
  emu_k_range(s, (int)(unit / (s.mt * s.nt)), kb0, kb1);
}

// Threads of both emulation kernels: warps 0-3 (producer, MMA issuer, two idle),
// one on each SM quarter, and the epilogue warps 4-11, two on each quarter.
constexpr int kPairThreads = 384;
// Registers per thread the kernels' register split assumes at launch: the
// register file is split by SM quarter, and on each quarter the control warp's
// 56 plus two epilogue warps' 224 must fit in the three warps' launch share,
// 56 + 2 x 224 = 3 x 168.
constexpr int kPairMinRegs = 168;

struct ELayout {
  static constexpr int NACC = 512 / EBN;                        // accumulator buffers
  static constexpr int A_BYTES = EBM * EBK * 2;
  static constexpr int B_BYTES = EBN * EBK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int BAR_OFF = ESTAGES * STAGE_BYTES;
  static constexpr int NBARS = 2 * ESTAGES + 2 * NACC + 1;      // full, empty, tfull, tempty, drain
  static constexpr int TOTAL = BAR_OFF + NBARS * 8 + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};

__global__ void __launch_bounds__(kPairThreads, 1)
emu_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                EmuArgs a) {
  using L = ELayout;
  constexpr int NACC = L::NACC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + ESTAGES;
  uint64_t* tfull = empty + ESTAGES;
  uint64_t* tempty = tfull + NACC;
  uint64_t* drain = tempty + NACC;
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

  // register split per SM quarter, as in the pair kernel
  if (warp >= 4) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 224;\n" ::: "memory");
    uint32_t te[NACC];
#pragma unroll
    for (int b = 0; b < NACC; ++b) te[b] = tc::mapa_shared(&tempty[b], 0);
    emu_fx_epilogue<EBN, EBM, 4>(a, cta, nunits, 0, tmem_base, tfull, te, w, warp, lane);
  } else {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 56;\n" ::: "memory");
  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0, armed = 0, armed_ph = 0;
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        const Unit u = emu_unit_of_cta(a.sch, cta, ui);
        const bool ok = emu_walk(
            a, u.kb0, u.kb1, [] { return true; },
            [&](int q, int lvl, int64_t kb, bool) {
              if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) return false;
              tc::mbar_arrive_expect_tx(&full[stage], L::STAGE_BYTES);
              uint8_t* sa = smem + stage * L::STAGE_BYTES;
              tma_load_slice(sa, &tmA, &full[stage], kb, (int32_t)(u.tile_row * EBM), q - 1);
              tma_load_slice(sa + L::A_BYTES, &tmB, &full[stage], kb,
                             (int32_t)(u.tile_col * EBN), lvl - q - 1);
              armed |= 1u << stage;
              armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
              if (++stage == ESTAGES) { stage = 0; ph ^= 1; }
              return true;
            },
            [] {});
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
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        int64_t kb0, kb1;
        emu_unit_range(a.sch, cta, ui, kb0, kb1);
        const bool ok = emu_walk(
            a, kb0, kb1,
            [&] {
              if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) return false;
              tc::tc_fence_after();
              return true;
            },
            [&](int, int, int64_t, bool first) {
              if (!tc::mbar_wait(&full[stage], ph, w)) return false;
              tc::tc_fence_after();
              const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
              const uint32_t sb = sa + L::A_BYTES;
              const uint32_t d = tmem_base + acc * EBN;
#pragma unroll
              for (int kk = 0; kk < EBK / 16; ++kk)
                tc::mma_bf16(d, tc::smem_desc_sw128(sa + kk * 32),
                             tc::smem_desc_sw128(sb + kk * 32), idesc,
                             (first && kk == 0) ? 0u : 1u);
              tc::mma_commit(&empty[stage]);
              if (++stage == ESTAGES) { stage = 0; ph ^= 1; }
              return true;
            },
            [&] {
              tc::mma_commit(&tfull[acc]);
              aph[acc] ^= 1;
              acc = (acc + 1) == NACC ? 0 : acc + 1;
            });
        if (!ok) break;
      }
      tc::mma_commit(drain);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, 512);
  }
}

// ---- CTA-pair kernel ----------------------------------------------------------------
//
// A cluster of two CTAs computes a 256 x BN tile (BN = 256 or 128) with
// tcgen05.mma.cta_group::2 (M = 256, N = BN): each CTA loads its own 128 rows of
// the A slice and its own BN / 2 of the BN columns of the B slice (no multicast),
// the even CTA issues the MMAs and commits to the barriers of both, and each CTA
// drains its own 128 x BN accumulator.  N = 256 instructions run the tensor
// cores at their full rate per clock (N = 128 ones reach about 81 % of it), and
// per SM an MMA step reads 8 KB of operands for 128 x 256 x 16 products.
//
template <int BN>
struct PairLayout {
  static constexpr int NACC = 512 / BN;                   // accumulator buffers
  static constexpr int A_BYTES = EBM * EBK * 2;           // own 128 rows
  static constexpr int B_BYTES = (BN / 2) * EBK * 2;      // own BN / 2 columns
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = BN == 256 ? 7 : 9;
  static constexpr int BAR_OFF = STAGES * STAGE_BYTES;
  // full, empty, tfull, tempty, drain, peer-count exchange
  static constexpr int NBARS = 2 * STAGES + 2 * NACC + 2;
  static constexpr int TOTAL = BAR_OFF + NBARS * 8 + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};

__device__ __forceinline__ void tma_load_slice_pair(void* dst, const CUtensorMap* map,
                                                    uint32_t bar_cluster, int64_t kb, int32_t y,
                                                    int32_t q) {
  const int64_t t = kb * EBK;
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];\n" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"((int32_t)(t % EKB)), "r"(y),
      "r"((int32_t)(t / EKB)), "r"(q)
      : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kPairThreads, 1)
emu_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                EmuArgs a) {
  using L = PairLayout<BN>;
  constexpr int S = L::STAGES;
  constexpr int NACC = L::NACC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + NACC;
  uint64_t* drain = tempty + NACC;
  uint64_t* xchg = drain + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(xchg + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  uint32_t* peer_issued = tslot + 2;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = tc::cluster_ctarank();
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);   // leader: its producer's arrival + both CTAs' bytes
      tc::mbar_init(&empty[s], 1);  // the leader's commit, multicast to both CTAs
    }
    for (int b = 0; b < NACC; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 16);  // leader: the 8 epilogue warps of each CTA
    }
    tc::mbar_init(drain, 1);
    tc::mbar_init(xchg, 1);  // leader: the odd CTA's count of issued stages
    *abort_flag = 0;
    *peer_issued = 0;
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

  // Register split: the control warps give registers back to the epilogue warps
  // on their own SM quarter (warp w runs on quarter w % 4); the epilogue threads
  // hold BN / 2 level sums each.  The launch provides kPairMinRegs per thread
  // (the host checks before launching).
  if (warp >= 4) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 224;\n" ::: "memory");
    uint32_t te[NACC];
#pragma unroll
    for (int b = 0; b < NACC; ++b) te[b] = tc::mapa_shared(&tempty[b], 0);
    emu_fx_epilogue<BN, 2 * EBM, 4>(a, pair, nunits, (int64_t)rank * EBM, tmem_base, tfull, te,
                                    w, warp, lane);
  } else {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 56;\n" ::: "memory");
  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0;
      uint32_t issued = 0;  // stages whose copies this CTA issued
      uint32_t full_cl[S];
#pragma unroll
      for (int s = 0; s < S; ++s) full_cl[s] = tc::mapa_shared(&full[s], 0);
      // Lock-step super-chunks (cooperative launches only): the leader's producer
      // of every pair counts each super-chunk it starts on a global counter and
      // starts super-chunk g (in the order rounds x super-chunks) only once every
      // pair has started g - 1, so concurrent pairs stream the same slice panels
      // through L2.  A pair without a unit in a round counts that round's
      // super-chunks at once.
      // With a k split, every unit counts as many super-chunks as the longest k
      // slice has; a shorter one counts the rest at its end.
      const int npairs = (int)(gridDim.x >> 1);
      const int64_t total = a.sch.mt * a.sch.nt * a.sch.pk;
      const int64_t rounds = a.lockstep ? (total + npairs - 1) / npairs : nunits;
      const int64_t nch = cdiv64(cdiv64(a.sch.kbt, a.chunk_kb), a.sch.pk);
      auto chunk_tick = [&](int64_t g) -> bool {
        if (!(a.lockstep && leader)) return true;
        if (g >= 1) {
          const unsigned int want = (unsigned int)(g * npairs);
          const long long t0 = clock64();
          while (*reinterpret_cast<volatile unsigned int*>(a.lockstep) < want) {
            if (*abort_flag) return false;
            if (clock64() - t0 > w.limit) {
              atomicCAS(a.status, 0, (int)COSMA_ERR_TIMEOUT);
              *abort_flag = 1;
              return false;
            }
            __nanosleep(128);
          }
          __threadfence();
        }
        atomicAdd(a.lockstep, 1u);
        return true;
      };
      for (int64_t ui = 0; ui < rounds && !*abort_flag; ++ui) {
        if (ui >= nunits) {
          if (a.lockstep && leader) atomicAdd(a.lockstep, (unsigned int)nch);
          continue;
        }
        const Unit u = emu_unit_of_cta(a.sch, pair, ui);
        const bool ok = emu_walk_chunks(
            a, u.kb0, u.kb1, [&](int64_t c) { return chunk_tick(ui * nch + c); },
            [] { return true; },
            [&](int q, int lvl, int64_t kb, bool) {
              if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) return false;
              if (leader) tc::mbar_arrive_expect_tx(&full[stage], 2 * L::STAGE_BYTES);
              uint8_t* sa = smem + stage * L::STAGE_BYTES;
              tma_load_slice_pair(sa, &tmA, full_cl[stage], kb,
                                  (int32_t)(u.tile_row * (2 * EBM) + rank * EBM), q - 1);
              tma_load_slice_pair(sa + L::A_BYTES, &tmB, full_cl[stage], kb,
                                  (int32_t)(u.tile_col * BN + rank * (BN / 2)), lvl - q - 1);
              ++issued;
              if (++stage == S) { stage = 0; ph ^= 1; }
              return true;
            },
            [] {});
        if (!ok) break;
        const int64_t used = cdiv64(u.kb1 - u.kb0, a.chunk_kb);
        if (a.lockstep && leader && used < nch) atomicAdd(a.lockstep, (unsigned int)(nch - used));
      }
      // The odd CTA's copies signal the leader's barriers: it reports how many
      // stages it issued, and on an abort the leader waits (bounded) until every
      // stage either CTA may still have in flight has landed, so neither CTA
      // leaves (final cluster barrier) with a copy still writing into it.
      if (*abort_flag) tc::st_cluster_u32(tc::mapa_shared(const_cast<int*>(abort_flag), rank ^ 1), 1u);
      if (!leader) {
        tc::st_cluster_u32(tc::mapa_shared(peer_issued, 0), issued);
        tc::mbar_arrive_remote(tc::mapa_shared(xchg, 0));
      } else if (*abort_flag) {
        const long long t0 = clock64();
        bool got = false;
        while (!(got = tc::mbar_try_wait_cluster(xchg, 0)) && clock64() - t0 < tc::kDrainCycles) {
        }
        if (got) {
          const uint32_t n0 = issued, n1 = *reinterpret_cast<volatile uint32_t*>(peer_issued);
          const uint32_t top = n0 > n1 ? n0 : n1;
          for (uint32_t i = top > (uint32_t)S ? top - S : 0u; i < top; ++i) {
            const int s = (int)(i % S);
            const uint32_t par = (i / S) & 1u;
            if (i >= n0) tc::mbar_arrive_expect_tx(&full[s], L::STAGE_BYTES);  // only the peer's
            else if (i >= n1) tc::mbar_complete_tx(&full[s], L::STAGE_BYTES);  // the peer's never come
            const long long t1 = clock64();
            while (!tc::mbar_try_wait(&full[s], par) && clock64() - t1 < tc::kDrainCycles) {
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (leader && tc::elect_one()) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(2 * EBM, BN);
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[NACC];
#pragma unroll
      for (int b = 0; b < NACC; ++b) aph[b] = 0;
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        int64_t kb0, kb1;
        emu_unit_range(a.sch, pair, ui, kb0, kb1);
        const bool ok = emu_walk(
            a, kb0, kb1,
            [&] {
              if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) return false;
              tc::tc_fence_after();
              return true;
            },
            [&](int, int, int64_t, bool first) {
              if (!tc::mbar_wait(&full[stage], ph, w)) return false;
              tc::tc_fence_after();
              const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
              const uint32_t sb = sa + L::A_BYTES;
              const uint32_t d = tmem_base + acc * BN;
#pragma unroll
              for (int kk = 0; kk < EBK / 16; ++kk)
                tc::mma_bf16_pair(d, tc::smem_desc_sw128(sa + kk * 32),
                                  tc::smem_desc_sw128(sb + kk * 32), idesc,
                                  (first && kk == 0) ? 0u : 1u);
              tc::mma_commit_pair(&empty[stage]);
              if (++stage == S) { stage = 0; ph ^= 1; }
              return true;
            },
            [&] {
              tc::mma_commit_pair(&tfull[acc]);
              aph[acc] ^= 1;
              acc = (acc + 1) == NACC ? 0 : acc + 1;
            });
        if (!ok) break;
      }
      tc::mma_commit_pair(drain);  // every MMA of the pair done (both CTAs' drain barriers)
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  }
  }
  __syncthreads();
  tc::tc_fence_before();
  tc::cluster_sync();  // no CTA leaves while its peer may still signal its barriers
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc_pair(tmem_base, 512);
}

// k-split plans: C = alpha X 2^(sigma_i + tau_j + eoff) + beta_c C from the summed
// exact totals X [m][n] -- the arithmetic of the kernels' own FP64 store, in the
// same order, so a split changes no bit of C.
__global__ void emu_finish_kernel(const long long* __restrict__ X, int64_t m, int64_t n,
                                  const int* __restrict__ eA, const int* __restrict__ eB, int eoff,
                                  double alpha, double beta_c, double* C, int64_t ldc) {
  for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
    const int ea = eA[i];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
      const int eb = eB[j];
      double x = (ea == kExpNone || eb == kExpNone) ? 0.0
                                                    : scale_pow2((double)X[i * n + j], ea + eb + eoff);
      if (alpha != 1.0) x *= alpha;
      double* dst = C + i * ldc + j;
      if (beta_c != 0.0) x = fma(beta_c, *dst, x);
      *dst = x;
    }
  }
}

// 4-D map over the k-blocked slices of `rows` rows starting at `base` (a row
// block of an operand with slice_rows rows): dims (EKB, rows, panels, slices).
int encode_tmap_slices(CUtensorMap* map, const void* base, int64_t rows, int64_t k, int s,
                       int64_t slice_rows, int box_rows) {
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
  const int64_t nkb = emu_kpad(k) / EKB;
  cuuint64_t dims[4] = {(cuuint64_t)EKB, (cuuint64_t)rows, (cuuint64_t)nkb, (cuuint64_t)s};
  cuuint64_t strides[3] = {(cuuint64_t)(EKB * 2), (cuuint64_t)(slice_rows * EKB * 2),
                           (cuuint64_t)(nkb * slice_rows * EKB * 2)};
  cuuint32_t box[4] = {(cuuint32_t)EBK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

}  // namespace

int64_t emu_padded_k(int64_t k) { return emu_kpad(k); }

namespace {
// split_a_kernel grid: x covers kpad in 1024-column groups, y enough rows to fill
// the GPU (the kernel strides over the rest).
dim3 split_a_grid(int64_t rows, int64_t kpad) {
  const int64_t gx = (kpad + 1023) / 1024;
  int64_t gy = (152LL * 16 + gx - 1) / gx;
  if (gy > rows) gy = rows;
  if (gy > 65535) gy = 65535;
  if (gy < 1) gy = 1;
  return dim3((unsigned)gx, (unsigned)gy);
}
}  // namespace

namespace {
// Bytes of the kernels' running totals: one 128 x 256 int64 region per CTA of the
// largest pair grid the problem can use (a single-SM CTA's 128 x 128 region is
// half of one) -- with a k split, of the largest grid the device allows.
int64_t emu_total_bytes(int64_t m, int64_t n, int sms, bool split) {
  const int64_t tiles = ((m + 2 * EBM - 1) / (2 * EBM)) * ((n + EBN - 1) / EBN);
  const int64_t pairs = split ? std::max(1, sms / 2)
                              : std::min<int64_t>(std::max(1, sms / 2), std::max<int64_t>(tiles, 1));
  return rup(2 * pairs * (int64_t)EBM * 256 * 8, 256);
}
}  // namespace

long long emu_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_config& cfg,
                              int sms, int64_t split_elems) {
  const int s = emu_slices(cfg);
  const int64_t kp = emu_kpad(k);
  return rup(m * 4, 256) + rup(n * 4, 256) + rup((int64_t)s * m * kp * 2, 256) +
         rup((int64_t)s * n * kp * 2, 256) + emu_total_bytes(m, n, sms, split_elems > 0) +
         rup(split_elems * 8, 256) + 256;
}

EmuWorkspace emu_carve(void* ws, int64_t m, int64_t n, int64_t k, const cosma_config& cfg,
                       int sms, int64_t split_elems) {
  const int s = emu_slices(cfg);
  const int64_t kp = emu_kpad(k);
  uint8_t* w = static_cast<uint8_t*>(ws);
  EmuWorkspace e;
  e.eA = reinterpret_cast<int*>(w);
  w += rup(m * 4, 256);
  e.eB = reinterpret_cast<int*>(w);
  w += rup(n * 4, 256);
  e.SA = w;
  w += rup((int64_t)s * m * kp * 2, 256);
  e.SB = w;
  w += rup((int64_t)s * n * kp * 2, 256);
  e.T = reinterpret_cast<long long*>(w);
  e.t_bytes = emu_total_bytes(m, n, sms, split_elems > 0);
  w += e.t_bytes;
  e.X = split_elems > 0 ? reinterpret_cast<long long*>(w) : nullptr;
  w += rup(split_elems * 8, 256);
  e.lockstep = reinterpret_cast<unsigned int*>(w);
  e.row_pitch = EKB;
  return e;
}

int emu_check_config(const cosma_config& cfg) {
  const int s = emu_slices(cfg), beta = emu_bits(cfg);
  if (s < 2 || s > EMU_MAX_SLICES || beta < 2 || beta > 8 || beta * s - 1 > 62)
    return COSMA_ERR_INVALID_ARG;
  return COSMA_OK;
}

int emu_prepare_a(const double* A, int64_t m, int64_t k, int64_t lda, int trans, int* eA,
                  void* SA, int64_t slice_rows, int* status, const cosma_config& cfg,
                  cudaStream_t st) {
  const int s = emu_slices(cfg), beta = emu_bits(cfg);
  const int64_t kp = emu_kpad(k);
  if (m <= 0) return COSMA_OK;
  if (trans) {  // A stored as k x m: its rows are columns of the stored matrix
    if ((kp + 31) / 32 > 65535) return COSMA_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(eA, 0x80, (size_t)m * 4, st) != cudaSuccess)
      return (int)cudaGetLastError();
    dim3 g1((unsigned)((m + 255) / 256), (unsigned)((k + 255) / 256));
    col_exp_kernel<<<g1, 256, 0, st>>>(A, k, m, lda, eA, status);
    count_launch();
    dim3 g2((unsigned)((m + 31) / 32), (unsigned)((kp + 31) / 32));
    split_b_kernel<<<g2, dim3(32, 8), 0, st>>>(A, k, m, lda, eA, static_cast<__nv_bfloat16*>(SA),
                                               kp, slice_rows, s, beta);
    count_launch();
    return (int)cudaGetLastError();
  }
  const int64_t rb = m < 65535LL * 16 ? m : 65535LL * 16;
  row_exp_kernel<<<(unsigned)rb, 256, 0, st>>>(A, m, k, lda, eA, status);
  count_launch();
  split_a_kernel<<<split_a_grid(m, kp), 256, 0, st>>>(A, m, k, lda, eA,
                                                      static_cast<__nv_bfloat16*>(SA), kp,
                                                      slice_rows, s, beta);
  count_launch();
  return (int)cudaGetLastError();
}

int emu_prepare_b(const double* B, int64_t k, int64_t n, int64_t ldb, int trans, int* eB,
                  void* SB, int64_t slice_rows, int* status, const cosma_config& cfg,
                  cudaStream_t st) {
  const int s = emu_slices(cfg), beta = emu_bits(cfg);
  const int64_t kp = emu_kpad(k);
  if (n <= 0) return COSMA_OK;
  if (trans) {  // B stored as n x k: its columns are rows of the stored matrix
    const int64_t rb = n < 65535LL * 16 ? n : 65535LL * 16;
    row_exp_kernel<<<(unsigned)rb, 256, 0, st>>>(B, n, k, ldb, eB, status);
    count_launch();
    split_a_kernel<<<split_a_grid(n, kp), 256, 0, st>>>(B, n, k, ldb, eB,
                                                        static_cast<__nv_bfloat16*>(SB), kp,
                                                        slice_rows, s, beta);
    count_launch();
    return (int)cudaGetLastError();
  }
  if ((kp + 31) / 32 > 65535) return COSMA_ERR_UNSUPPORTED;
  if (cudaMemsetAsync(eB, 0x80, (size_t)n * 4, st) != cudaSuccess) return (int)cudaGetLastError();
  dim3 g1((unsigned)((n + 255) / 256), (unsigned)((k + 255) / 256));
  col_exp_kernel<<<g1, 256, 0, st>>>(B, k, n, ldb, eB, status);
  count_launch();
  dim3 g2((unsigned)((n + 31) / 32), (unsigned)((kp + 31) / 32));
  split_b_kernel<<<g2, dim3(32, 8), 0, st>>>(B, k, n, ldb, eB, static_cast<__nv_bfloat16*>(SB),
                                             kp, slice_rows, s, beta);
  count_launch();
  return (int)cudaGetLastError();
}

int emu_multiply(int64_t m, int64_t n, int64_t k, const cosma_plan& p, const cosma_config& cfg,
                 const int* eA, const void* SA, int64_t a_slice_rows, const int* eB,
                 const void* SB, int64_t b_slice_rows, double* C, int64_t ldc, double alpha,
                 double beta_c, long long* T, int64_t t_bytes, long long* X,
                 unsigned int* lockstep, int* status, long long wait_limit, cudaStream_t st) {
  const int s = emu_slices(cfg), beta = emu_bits(cfg);
  const Sched sch = sched_from_plan(m, n, k, p);
  const bool pairs = sch.tile_m == 2 * EBM;
  if (pairs ? (sch.tile_n != 256 && sch.tile_n != 128) : (sch.tile_m != EBM || sch.tile_n != EBN))
    return COSMA_ERR_INVALID_ARG;
  // order 1, k slices of whole super-chunks, a total to sum them in
  if (sch.k_block != EBK || sch.order != 1 || sch.pk < 1 ||
      sch.pk > cdiv64(sch.kbt, kEmuChunkKb) || (sch.pk > 1 && !X))
    return COSMA_ERR_INVALID_ARG;
  // the running totals: one 128 x tile_n int64 region per CTA of the launch
  if (!T || (pairs ? 2LL * sch.ctas : (long long)sch.ctas) > (long long)p.sms ||
      (pairs ? 2LL : 1LL) * sch.ctas * EBM * sch.tile_n * 8 > t_bytes)
    return COSMA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(C) & 7) return COSMA_ERR_INVALID_ARG;
  // COSMA_EMU_LOCKSTEP in the environment (read once): unset or 1 = lock-step
  // rounds under a cooperative launch; 0 = pairs free; 2 = lock-step rounds under
  // a plain cluster launch, for profilers that cannot launch cooperative cluster
  // kernels -- it relies on the one-pair-per-two-SMs grid being resident, and a
  // pair that is not would only make the others' bounded waits expire (status
  // COSMA_ERR_TIMEOUT), never hang.
  static const int lockstep_mode = [] {
    const char* e = getenv("COSMA_EMU_LOCKSTEP");
    return e && e[0] == '0' ? 0 : (e && e[0] == '2' ? 2 : 1);
  }();
  unsigned int* lockstep_counter =
      lockstep_mode != 0 && 2 * sch.ctas <= p.sms ? lockstep : nullptr;

  CUtensorMap ta, tb;
  int rc = encode_tmap_slices(&ta, SA, m, k, s, a_slice_rows, EBM);
  if (rc != COSMA_OK) return rc;
  rc = encode_tmap_slices(&tb, SB, n, k, s, b_slice_rows, pairs ? sch.tile_n / 2 : EBN);
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
  args.C = C;
  args.ldc = ldc;
  args.status = status;
  args.wait_limit = wait_limit;
  args.lockstep = nullptr;
  args.alpha = alpha;
  args.beta_c = beta_c;
  // Super-chunk: every level sum of a chunk must fit in int32 exactly (at most s
  // pairs x chunk x 2^(2 beta - 2)).  Each chunk ends in ceil(s / 2) merges of the
  // running total (levels in pairs), which are L2 reductions; 4096 k -- fewer
  // merges beat keeping a chunk's slice panels in L2 across the levels (one GB300,
  // 256 x 256 pair tiles, one merge per level, square 16384^3: 512 k 66.2, 1024 k
  // 72.6, 2048 k 77.6, 4096 k 78.3-79.6, 16384 k 80.3 TFLOP/s; largeK 4096 x 4096
  // x 2^20: 4096 k 64.3, 16384 k 62.7).
  // (With at most 12 slices of at most 8 bits the bound is above 10000 k, so
  // every accepted configuration uses the 4096-k super-chunk the planner assumes.)
  {
    // (a level's sum also takes the carry of the level below: at most 2^-beta of
    // that one's bound, plus one)
    const double lim =
        2147483646.0 / ((double)s * std::ldexp(1.0, 2 * beta - 2) * (1.0 + std::ldexp(1.0, -beta)));
    if ((double)kEmuChunkKb * EBK > lim) return COSMA_ERR_UNSUPPORTED;
    args.chunk_kb = kEmuChunkKb;
  }
  args.X = sch.pk > 1 ? X : nullptr;
  // Fixed-point base of the running total: every super-chunk adds
  // at most sum_{l=2}^{s+1} (l - 1) chunk 2^(2 beta - 2) 2^(beta (s + 1 - l)); the
  // smallest base that keeps the sum over all chunks below 2^62.
  args.T = T;
  {
    double per_chunk = 0.0;
    for (int l = 2; l <= s + 1; ++l)
      per_chunk += (double)(l - 1) * std::ldexp(1.0, 2 * beta - 2 + beta * (s + 1 - l));
    per_chunk *= (double)args.chunk_kb * EBK;
    const double bound = per_chunk * (double)((sch.kbt + args.chunk_kb - 1) / args.chunk_kb);
    int base = 0;
    while (std::ldexp(bound, -base) >= std::ldexp(1.0, 62)) ++base;
    args.t_base = base;
  }
  if (args.X && cudaMemsetAsync(args.X, 0, (size_t)(m * n) * 8, st) != cudaSuccess)
    return (int)cudaGetLastError();
  cudaError_t le;
  if (pairs) {
    auto kern = sch.tile_n == 256 ? emu_pair_kernel<256> : emu_pair_kernel<128>;
    const int alloc = sch.tile_n == 256 ? PairLayout<256>::ALLOC : PairLayout<128>::ALLOC;
    {
      // the warps' register split draws on what the launch allocates
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return (int)cudaGetLastError();
      if (fa.numRegs < kPairMinRegs) return COSMA_ERR_UNSUPPORTED;
    }
    const cudaError_t attr2 =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, alloc);
    if (attr2 != cudaSuccess) return (int)attr2;
    cudaLaunchConfig_t cfgl = {};
    cfgl.gridDim = dim3((unsigned)(2 * sch.ctas));
    cfgl.blockDim = dim3(kPairThreads);
    cfgl.dynamicSmemBytes = alloc;
    cfgl.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfgl.attrs = at;
    // Lock-step rounds need every pair resident at once: launch cooperatively
    // (at most one CTA per SM here); without that guarantee run free.
    cfgl.numAttrs = lockstep_counter && lockstep_mode == 1 ? 2 : 1;
    args.lockstep = lockstep_counter;
    if (lockstep_counter &&
        cudaMemsetAsync(lockstep_counter, 0, sizeof(unsigned int), st) != cudaSuccess)
      return (int)cudaGetLastError();
    prof_mark(st, true);
    le = cudaLaunchKernelEx(&cfgl, kern, ta, tb, args);
    if (le != cudaSuccess && lockstep_counter) {
      cudaGetLastError();
      cfgl.numAttrs = 1;
      args.lockstep = nullptr;
      le = cudaLaunchKernelEx(&cfgl, kern, ta, tb, args);
    }
    prof_mark(st, false);
  } else {
    const cudaError_t attr = cudaFuncSetAttribute(
        emu_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ELayout::ALLOC);
    if (attr != cudaSuccess) return (int)attr;
    {
      cudaFuncAttributes fa;  // the warps' register split draws on what the launch allocates
      if (cudaFuncGetAttributes(&fa, emu_gemm_kernel) != cudaSuccess) return (int)cudaGetLastError();
      if (fa.numRegs < kPairMinRegs) return COSMA_ERR_UNSUPPORTED;
    }
    prof_mark(st, true);
    emu_gemm_kernel<<<sch.ctas, kPairThreads, ELayout::ALLOC, st>>>(ta, tb, args);
    prof_mark(st, false);
    le = cudaGetLastError();
  }
  if (le != cudaSuccess) return (int)le;
  count_launch();
  if (args.X) {
    const int64_t gx = std::min<int64_t>((n + 255) / 256, 1024);
    const int64_t gy = std::min<int64_t>(m, 65535);
    emu_finish_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(
        args.X, m, n, eA, eB, 2 - beta * (s + 1) + args.t_base, alpha, beta_c, C, ldc);
    count_launch();
  }
  return (int)cudaGetLastError();
}

int launch_emu_bf16(const GemmArgs& g, const cosma_plan& p, const cosma_config& cfg, void* ws,
                    long long ws_bytes, int* status, long long wait_limit, cudaStream_t st) {
  int rc = emu_check_config(cfg);
  if (rc != COSMA_OK) return rc;
  const int64_t m = g.m, n = g.n, k = g.k;
  const int64_t split = p.pk > 1 ? m * n : 0;
  if (emu_workspace_bytes(m, n, k, cfg, p.sms, split) > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
  if ((emu_kpad(k) + 31) / 32 > 65535) return COSMA_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(g.A) & 7) || (reinterpret_cast<uintptr_t>(g.B) & 7) ||
      (reinterpret_cast<uintptr_t>(g.C) & 7))
    return COSMA_ERR_INVALID_ARG;
  const EmuWorkspace e = emu_carve(ws, m, n, k, cfg, p.sms, split);
  rc = emu_prepare_a(static_cast<const double*>(g.A), m, k, g.lda, g.trans_a, e.eA, e.SA, m,
                     status, cfg, st);
  if (rc != 0) return rc;
  rc = emu_prepare_b(static_cast<const double*>(g.B), k, n, g.ldb, g.trans_b, e.eB, e.SB, n,
                     status, cfg, st);
  if (rc != 0) return rc;
  return emu_multiply(m, n, k, p, cfg, e.eA, e.SA, m, e.eB, e.SB, n, static_cast<double*>(g.C),
                      g.ldc, g.alpha, g.beta, e.T, e.t_bytes, e.X, e.lockstep, status, wait_limit,
                      st);
}

}  // namespace cosma

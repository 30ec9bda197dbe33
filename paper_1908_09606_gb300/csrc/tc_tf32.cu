// K-TF32X3: FP32 C = alpha A B + beta C from three TF32 products on the
// tensor cores (tcgen05.mma kind::tf32).  The schedule is the one of the other
// tensor-core paths -- the paper's sequential schedule per CTA (Listing 1,
// Sec. 5.2): a 128 x 128 C tile stays in fast memory while A and B k panels
// stream through a TMA-fed shared-memory ring, the producer fetching round
// t+1 while the tensor cores multiply round t (Sec. 7.3) -- over the work
// units of the plan (schedule.h).  The element format is not the paper's.
//
// Splitting (a pre-pass per operand): h = tf32(x) and l = tf32(x - h), both
// rounded to nearest, so x = h + l + e with |e| <= 2^-22 |x|, and
//     A B ~ A_h B_h + A_h B_l + A_l B_h,
// the dropped A_l B_l and split remainders staying below about 3 2^-22 |A||B|.
// The parts are written K-major and k-blocked, [2][kbt][rows][32] f32 (zero
// beyond k): one TMA box is then 128 contiguous rows of 128 bytes whatever k
// is (row-major parts at k = 2^20 would put every row of a box in its own page).
//
// Accumulation: the tensor cores' fp32 accumulator does not round to nearest,
// and over a long k the error drifts one way (about 1e-4 relative at k =
// 16384 in one accumulator).  So the k range of a unit is cut into segments
// of SEG k blocks, each accumulated from zero in tensor memory, and the
// epilogue warps add the finished segments into registers in fp32 round to
// nearest.  Two accumulators alternate: the tensor cores fill one segment
// while the epilogue drains the other.
//
// Stage (64 KB): the A_h, A_l, B_h, B_l tiles of one k block, 128 rows x 32
// f32 each (one 128-byte swizzled row per tile row), by four 4-D TMA copies.
// Warp roles as in K-BF16: warp 0 TMA, warp 1 tensor memory + MMA, warps 2-5
// segment sums and stores (warp w reads tensor-memory lanes 32 (w % 4) ..).
//
// Lock-step ticks (balanced-stripe plans under a cooperative launch): the k
// range of every unit is walked in ticks of TICK k blocks; each producer adds
// one to a global counter per tick and does not start tick T before the
// counter says the CTAs have, on average, finished tick T - WINDOW.  The
// CTAs of a wave then stream the same k slices of their part panels, which
// stay in L2 (a wave's panels over all of k do not: 413 MB at 16384^3).
#include <cuda.h>
#include <cuda_runtime.h>
#include <mutex>
#include <stdlib.h>
#include <string.h>

#include "tc_common.cuh"

namespace cosma {

namespace {

constexpr int TM = 128;    // tile rows: one tensor-memory lane per row
constexpr int TN = 128;    // tile columns: accumulator columns
constexpr int TK = 32;     // k per block: one 128-byte row of f32
constexpr int STAGES = 3;
constexpr int SEG = 2;     // k blocks per tensor-memory segment
constexpr int TICK = 32;   // k blocks per lock-step tick (1024 k)
constexpr int WINDOW = 2;  // ticks a producer may run ahead of the average

struct TfLayout {
  static constexpr int PART = TM * TK * 4;  // one part tile, 16 KB (TN == TM)
  static constexpr int STAGE_BYTES = 4 * PART;
  static constexpr int BAR_OFF = STAGES * STAGE_BYTES;
  static constexpr int NBARS = 2 * STAGES + 5;  // full, empty, tfull[2], tempty[2], drain
  static constexpr int TOTAL = BAR_OFF + NBARS * 8 + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};
static_assert(TN == TM, "A and B part tiles share one size");

struct TfArgs {
  Sched s;
  float* C;
  int64_t ldc;
  float* partial;  // pk > 1: pk slices of m x n (row pitch n)
  int* status;
  long long wait_limit;
  int vec_ok;      // destination rows 16-byte aligned
  float alpha, beta;
  unsigned int* lockstep;  // zeroed tick counter (all CTAs resident), else null
  int64_t rounds;          // lock-step: units per CTA rounded up over the grid
  int64_t ticks;           // lock-step: ticks per round
};

// x = hi + lo + e with hi = tf32(x), lo = tf32(x - hi) (round to nearest, ties
// away), |e| <= 2^-22 |x|; x - hi is exact in f32.  A non-finite hi has lo = 0,
// and a finite x whose rounding would overflow keeps its truncated hi.
__device__ __forceinline__ void tf32_parts(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  if (isinf(hi) && isfinite(x)) hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  if (!isfinite(hi)) {
    lo = 0.f;
    return;
  }
  uint32_t l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}

// Index of element (part q, row r, k index t) in the k-blocked parts array.
__device__ __forceinline__ int64_t part_index(int q, int64_t r, int64_t t, int64_t rows,
                                              int64_t kbt) {
  return (((int64_t)q * kbt + (t >> 5)) * rows + r) * TK + (t & 31);
}

// Parts of a rows x cols matrix (ld) in its own orientation (cols = k), zero
// for k <= t < 32 kbt.  Each thread step takes 4 consecutive k (16-byte loads
// when vec: X 16-byte aligned and ld a multiple of 4) and writes one 16-byte
// chunk of each part; four steps are loaded before any is converted, so each
// thread keeps 64 bytes in flight.
__global__ void tf32_split_rows(const float* __restrict__ X, int64_t rows, int64_t cols,
                                int64_t ld, float* __restrict__ P, int64_t kbt, int vec) {
  const int64_t q4 = kbt * (TK / 4);  // 4-element chunks per row
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* x = X + r * ld;
    for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < q4; c0 += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t t = 4 * (c0 + u * stride);
        if (vec && t + 4 <= cols) {
          v[u] = *reinterpret_cast<const float4*>(x + t);
        } else {
          v[u].x = t < cols ? x[t] : 0.f;
          v[u].y = t + 1 < cols ? x[t + 1] : 0.f;
          v[u].z = t + 2 < cols ? x[t + 2] : 0.f;
          v[u].w = t + 3 < cols ? x[t + 3] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t c = c0 + u * stride;
        if (c >= q4) break;
        const int64_t t = 4 * c;
        float4 h, l;
        tf32_parts(v[u].x, h.x, l.x);
        tf32_parts(v[u].y, h.y, l.y);
        tf32_parts(v[u].z, h.z, l.z);
        tf32_parts(v[u].w, h.w, l.w);
        *reinterpret_cast<float4*>(P + part_index(0, r, t, rows, kbt)) = h;
        *reinterpret_cast<float4*>(P + part_index(1, r, t, rows, kbt)) = l;
      }
    }
  }
}

// Parts of the transpose of a k x n matrix (ld): rows j < n, k index t, zero
// for k <= t < 32 kbt.  A block takes 32 k x 64 j through shared memory
// (grid.y = kbt): reads are 256-byte row segments of X, writes one 16-byte
// chunk per thread and part.
__global__ void tf32_split_transpose(const float* __restrict__ X, int64_t k, int64_t n,
                                     int64_t ld, float* __restrict__ P, int64_t kbt) {
  __shared__ float th[64][33], tl[64][33];
  const int64_t t0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 64;
  const int tid = threadIdx.y * 32 + threadIdx.x;  // 256 threads
  float v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {  // element (t0 + 4u + ty/2 .., j0 + 32 (ty & 1) + tx)
    const int r = 4 * u + (threadIdx.y >> 1);
    const int64_t t = t0 + r, j = j0 + 32 * (threadIdx.y & 1) + threadIdx.x;
    v[u] = (t < k && j < n) ? X[t * ld + j] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int r = 4 * u + (threadIdx.y >> 1);
    const int jj = 32 * (threadIdx.y & 1) + threadIdx.x;
    float hi, lo;
    tf32_parts(v[u], hi, lo);
    th[jj][r] = hi;
    tl[jj][r] = lo;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 2; ++u) {  // 64 rows j x 8 chunks of 4 t = 512 chunks per part
    const int id = tid + 256 * u;
    const int jj = id >> 3, tq = (id & 7) * 4;
    const int64_t j = j0 + jj;
    if (j < n) {
      const int64_t t = t0 + tq;
      *reinterpret_cast<float4*>(P + part_index(0, j, t, n, kbt)) =
          make_float4(th[jj][tq], th[jj][tq + 1], th[jj][tq + 2], th[jj][tq + 3]);
      *reinterpret_cast<float4*>(P + part_index(1, j, t, n, kbt)) =
          make_float4(tl[jj][tq], tl[jj][tq + 1], tl[jj][tq + 2], tl[jj][tq + 3]);
    }
  }
}

// One row of a finished tile: cols (<= TN) values to dst, alpha / beta applied
// when scale is set (beta != 0 reads dst).
__device__ __forceinline__ void store_tile_row(float* dst, int64_t cols, const float (&v)[TN],
                                               bool vec, bool scale, float alpha, float beta) {
  if (scale) {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      if (j >= cols) continue;
      float x = alpha * v[j];
      if (beta != 0.f) x = fmaf(beta, dst[j], x);
      dst[j] = x;
    }
    return;
  }
  if (vec && cols == TN) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int j = 0; j < TN / 4; ++j)
      d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    return;
  }
#pragma unroll
  for (int j = 0; j < TN; ++j)
    if (j < cols) dst[j] = v[j];
}

__global__ void __launch_bounds__(192, 1)
tf32x3_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmB, TfArgs a) {
  using L = TfLayout;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 4);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) tc::tmem_alloc(tslot, 2 * TN);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const tc::WaitCtx w{a.wait_limit, a.status, abort_flag};
  const int cta = blockIdx.x;
  const int64_t nunits = units_of_cta(a.s, cta);

  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0;
      uint32_t armed = 0;  // bit s: stage s armed at least once; last parity in armed_ph
      uint32_t armed_ph = 0;
      const bool lock = a.lockstep != nullptr;
      const int64_t rounds = lock ? a.rounds : nunits;
      const int64_t ticks = lock ? a.ticks : 1;
      bool ok = true;
      for (int64_t ui = 0; ui < rounds && ok && !*abort_flag; ++ui) {
        Unit u{};
        if (ui < nunits) u = unit_of_cta(a.s, cta, ui);
        const int32_t ya = (int32_t)(u.tile_row * TM), yb = (int32_t)(u.tile_col * TN);
        for (int64_t t = 0; t < ticks && ok; ++t) {
          if (lock) {
            const int64_t T = ui * ticks + t;
            if (T >= WINDOW) {
              const unsigned int want = (unsigned int)((T - WINDOW + 1) * gridDim.x);
              const long long t0 = clock64();
              while (*reinterpret_cast<volatile unsigned int*>(a.lockstep) < want) {
                if (*abort_flag) break;
                if (clock64() - t0 > w.limit) {
                  atomicCAS(a.status, 0, (int)COSMA_ERR_TIMEOUT);
                  *abort_flag = 1;
                  break;
                }
                __nanosleep(256);
              }
              if (*abort_flag) { ok = false; break; }
            }
          }
          int64_t kb_lo = u.kb0, kb_hi = u.kb1;  // the whole unit, or this tick of it
          if (ui >= nunits) kb_hi = kb_lo;
          if (lock) {
            kb_lo = u.kb0 + t * TICK;
            if (kb_lo > kb_hi) kb_lo = kb_hi;
            if (kb_lo + TICK < kb_hi) kb_hi = kb_lo + TICK;
          }
          for (int64_t kb = kb_lo; kb < kb_hi; ++kb) {
            if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) { ok = false; break; }
            tc::mbar_arrive_expect_tx(&full[stage], L::STAGE_BYTES);
            uint8_t* sa = smem + stage * L::STAGE_BYTES;
            const int32_t z = (int32_t)kb;
            tc::tma_load_4d(sa, &tmA, &full[stage], 0, ya, z, 0);                 // A_h
            tc::tma_load_4d(sa + L::PART, &tmA, &full[stage], 0, ya, z, 1);       // A_l
            tc::tma_load_4d(sa + 2 * L::PART, &tmB, &full[stage], 0, yb, z, 0);   // B_h
            tc::tma_load_4d(sa + 3 * L::PART, &tmB, &full[stage], 0, yb, z, 1);   // B_l
            armed |= 1u << stage;
            armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
            if (++stage == STAGES) { stage = 0; ph ^= 1; }
          }
          if (lock) atomicAdd(a.lockstep, 1u);
        }
      }
      if (*abort_flag) {
        // Let every copy this thread started land before shared memory is released.
        for (int s = 0; s < STAGES; ++s) {
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
      constexpr uint32_t idesc = tc::idesc_tf32_f32(TM, TN);
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[2] = {0, 0};
      bool ok = true;
      for (int64_t ui = 0; ui < nunits && ok && !*abort_flag; ++ui) {
        const Unit u = unit_of_cta(a.s, cta, ui);
        for (int64_t s0 = u.kb0; s0 < u.kb1 && ok; s0 += SEG) {
          const int64_t s1 = s0 + SEG < u.kb1 ? s0 + SEG : u.kb1;
          if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t d = tmem_base + acc * TN;
          for (int64_t kb = s0; kb < s1; ++kb) {
            if (!tc::mbar_wait(&full[stage], ph, w)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t ah = tc::smem_u32(smem + stage * L::STAGE_BYTES);
            const uint32_t al = ah + L::PART, bh = ah + 2 * L::PART, bl = ah + 3 * L::PART;
            // K = 8 tf32 (32 bytes of each 128-byte row) per instruction; the two
            // small products first, then the leading one
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_tf32(d, tc::smem_desc_sw128(al + kk * 32), tc::smem_desc_sw128(bh + kk * 32),
                           idesc, (kb > s0 || kk > 0) ? 1u : 0u);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_tf32(d, tc::smem_desc_sw128(ah + kk * 32), tc::smem_desc_sw128(bl + kk * 32),
                           idesc, 1u);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_tf32(d, tc::smem_desc_sw128(ah + kk * 32), tc::smem_desc_sw128(bh + kk * 32),
                           idesc, 1u);
            tc::mma_commit(&empty[stage]);
            if (++stage == STAGES) { stage = 0; ph ^= 1; }
          }
          if (!ok) break;
          tc::mma_commit(&tfull[acc]);
          aph[acc] ^= 1;
          acc ^= 1;
        }
      }
      // All MMAs of this thread complete before tensor memory is released.
      tc::mma_commit(drain);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  } else {
    const int q = warp & 3;  // tensor-memory lane quadrant this warp may access
    uint32_t acc = 0;
    uint32_t tph[2] = {0, 0};
    bool ok = true;
    for (int64_t ui = 0; ui < nunits && ok; ++ui) {
      const Unit u = unit_of_cta(a.s, cta, ui);
      float sum[TN];
#pragma unroll
      for (int j = 0; j < TN; ++j) sum[j] = 0.f;
      for (int64_t s0 = u.kb0; s0 < u.kb1; s0 += SEG) {
        if (!tc::mbar_wait(&tfull[acc], tph[acc], w)) { ok = false; break; }
        tc::tc_fence_after();
#pragma unroll
        for (int c = 0; c < TN / 32; ++c) {
          uint32_t r[32];
          tc::tmem_ld_32x32(tmem_base + ((uint32_t)(q * 32) << 16) + acc * TN + c * 32, r);
          tc::tmem_wait_ld_r32(r);  // r is read only after the wait
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[c * 32 + j] += __uint_as_float(r[j]);
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[acc]);
        tph[acc] ^= 1;
        acc ^= 1;
      }
      if (!ok) break;
      const int64_t row = u.tile_row * TM + q * 32 + lane;
      const int64_t col0 = u.tile_col * TN;
      if (row < a.s.m && col0 < a.s.n) {
        const int64_t cols = a.s.n - col0 < TN ? a.s.n - col0 : TN;
        if (a.s.pk > 1)
          store_tile_row(a.partial + (int64_t)u.ks * a.s.m * a.s.n + row * a.s.n + col0, cols,
                         sum, (a.s.n & 3) == 0, false, 1.f, 0.f);
        else
          store_tile_row(a.C + row * a.ldc + col0, cols, sum, a.vec_ok != 0,
                         a.alpha != 1.f || a.beta != 0.f, a.alpha, a.beta);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, 2 * TN);
  }
}

inline int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

}  // namespace

long long tf32x3_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_plan& p) {
  const int64_t kpad = round_up(k, TK);
  long long b = 0;
  if (p.pk > 1) b += round_up((long long)p.pk * m * n * 4, 256);
  b += round_up(2 * m * kpad * 4, 256) + round_up(2 * n * kpad * 4, 256);
  return b + 256;  // lock-step tick counter
}

// Splits A and B into K-major TF32 parts in the workspace, then runs the
// three-product kernel over the plan's units and, when k is split, the Reduce.
int launch_tc_tf32x3(const GemmArgs& g, const Sched& s, const cosma_plan& p, void* ws,
                     long long ws_bytes, int* status, long long wait_limit, cudaStream_t st) {
  if (p.tile_m != TM || p.tile_n != TN || p.k_block != TK) return COSMA_ERR_INVALID_ARG;
  const int64_t kbt = (g.k + TK - 1) / TK, kpad = kbt * TK;
  if (tf32x3_workspace_bytes(g.m, g.n, g.k, p) > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
  if (kbt > 65535) return COSMA_ERR_UNSUPPORTED;  // split grids' y extent
  uint8_t* w = static_cast<uint8_t*>(ws);
  long long off = 0;
  float* partial = nullptr;
  if (p.pk > 1) {
    partial = reinterpret_cast<float*>(w + off);
    off += round_up((long long)p.pk * g.m * g.n * 4, 256);
  }
  float* PA = reinterpret_cast<float*>(w + off);
  off += round_up(2 * g.m * kpad * 4, 256);
  float* PB = reinterpret_cast<float*>(w + off);
  off += round_up(2 * g.n * kpad * 4, 256);
  unsigned int* counter = reinterpret_cast<unsigned int*>(w + off);
  const float* A = static_cast<const float*>(g.A);
  const float* B = static_cast<const float*>(g.B);
  // rows kernel: x covers a row's 4-element chunks (4 per thread per pass, at most 8
  // blocks), y the rows
  auto rows_grid = [kpad](int64_t rows) {
    int64_t x = (kpad / 4 + 1023) / 1024;
    if (x > 8) x = 8;
    const int64_t y = rows < 8192 ? rows : 8192;
    return dim3((unsigned)(x < 1 ? 1 : x), (unsigned)(y < 1 ? 1 : y));
  };
  auto t_grid = [kbt](int64_t n) { return dim3((unsigned)((n + 63) / 64), (unsigned)kbt); };
  auto vec_of = [](const float* X, int64_t ld) {
    return ((reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ld & 3) == 0) ? 1 : 0;
  };
  // A parts: A row by row, or the transpose of a stored k x m
  if (!g.trans_a)
    tf32_split_rows<<<rows_grid(g.m), 256, 0, st>>>(A, g.m, g.k, g.lda, PA, kbt,
                                                    vec_of(A, g.lda));
  else
    tf32_split_transpose<<<t_grid(g.m), dim3(32, 8), 0, st>>>(A, g.k, g.m, g.lda, PA, kbt);
  count_launch();
  // B parts: the transpose of B, or a stored n x k row by row
  if (!g.trans_b)
    tf32_split_transpose<<<t_grid(g.n), dim3(32, 8), 0, st>>>(B, g.k, g.n, g.ldb, PB, kbt);
  else
    tf32_split_rows<<<rows_grid(g.n), 256, 0, st>>>(B, g.n, g.k, g.ldb, PB, kbt,
                                                    vec_of(B, g.ldb));
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;

  CUtensorMap ta, tb;
  int rc = encode_tmap_f32_parts(&ta, PA, g.m, kbt, TM);
  if (rc != COSMA_OK) return rc;
  rc = encode_tmap_f32_parts(&tb, PB, g.n, kbt, TN);
  if (rc != COSMA_OK) return rc;
  TfArgs args;
  args.s = s;
  args.C = static_cast<float*>(g.C);
  args.ldc = g.ldc;
  args.partial = partial;
  args.status = status;
  args.wait_limit = wait_limit;
  args.vec_ok = ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0 && (g.ldc & 3) == 0) ? 1 : 0;
  args.alpha = (float)g.alpha;
  args.beta = (float)g.beta;
  args.lockstep = nullptr;
  args.rounds = 0;
  args.ticks = 0;

  // Lock-step ticks need every CTA resident at once: balanced-stripe plans with
  // at most one CTA per SM, launched cooperatively.  COSMA_TF32_LOCKSTEP=0 runs
  // the CTAs free; =2 keeps the ticks under a plain launch (for profilers that
  // cannot launch cooperative kernels: every CTA is resident there too, and
  // every wait is bounded).
  static const int lockstep_mode = [] {
    const char* v = getenv("COSMA_TF32_LOCKSTEP");
    return v && v[0] == '0' ? 0 : (v && v[0] == '2' ? 2 : 1);
  }();
  if (lockstep_mode != 0 && s.order == 1 && s.ctas <= p.sms) {
    const int64_t rounds = (s.mt * s.nt * s.pk + s.ctas - 1) / s.ctas;
    const int64_t ticks = ((s.kbt + s.pk - 1) / s.pk + TICK - 1) / TICK;
    if (rounds * ticks * s.ctas < (1LL << 31)) {
      args.lockstep = counter;
      args.rounds = rounds;
      args.ticks = ticks;
      if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess)
        return (int)cudaGetLastError();
    }
  }

  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(tf32x3_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TfLayout::ALLOC);
  });
  if (attr != cudaSuccess) return (int)attr;
  cudaLaunchConfig_t cfgl = {};
  cfgl.gridDim = dim3((unsigned)s.ctas);
  cfgl.blockDim = dim3(192);
  cfgl.dynamicSmemBytes = TfLayout::ALLOC;
  cfgl.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfgl.attrs = at;
  cfgl.numAttrs = args.lockstep && lockstep_mode == 1 ? 1 : 0;
  prof_mark(st, true);
  e = cudaLaunchKernelEx(&cfgl, tf32x3_gemm_kernel, ta, tb, args);
  if (e != cudaSuccess && args.lockstep) {
    // not launchable cooperatively: run the CTAs free
    cudaGetLastError();
    cfgl.numAttrs = 0;
    args.lockstep = nullptr;
    e = cudaLaunchKernelEx(&cfgl, tf32x3_gemm_kernel, ta, tb, args);
  }
  prof_mark(st, false);
  count_launch();
  if (e != cudaSuccess) return (int)e;
  if (p.pk > 1) return launch_reduce(COSMA_F32, g, p.pk, partial, st);
  return 0;
}

}  // namespace cosma

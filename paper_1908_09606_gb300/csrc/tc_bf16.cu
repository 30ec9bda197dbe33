// K-BF16: C (f32) = A (bf16) B (bf16) on the 5th-generation tensor cores.
//
// The paper's sequential schedule (Listing 1, Sec. 5.2) per CTA: a 128 x BN C
// tile is held in tensor memory (the accumulator never leaves fast memory
// until the tile is done), while A-column panels (128 x 64) and B-row panels
// (64 x BN) stream through a STAGES-deep shared-memory ring filled by TMA --
// Alg. 1's DistrData + Multiply with the double buffering of Sec. 7.3 (the
// producer fetches round t+1 while the tensor cores multiply round t).
//
// Warp roles (192 threads): warp 0 issues TMA loads, warp 1 allocates tensor
// memory and issues tcgen05.mma, warps 2-5 drain finished accumulators
// (tcgen05.ld) to global memory.  Two accumulators alternate so the epilogue
// of one tile overlaps the main loop of the next.  Work units come from the
// plan's schedule (schedule.h); a k split writes f32 partials that the
// Reduce kernel sums in a fixed order.
//
// B arrives row-major (k x n, n contiguous).  When its rows are 16-byte aligned
// it is loaded as it is -- 64 x 64 TMA boxes (64 n by 64 k, 128-byte swizzle) --
// and multiplied as an MN-major operand; otherwise it is first transposed into
// the workspace so both operands are K-major.  A is loaded in place unless its
// rows are at least 256 KB apart (then through a k-blocked copy, so one box is
// contiguous) or not 16-byte aligned (then through a pitch-padded copy).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mutex>
#include <string.h>

#include "tc_common.cuh"

namespace cosma {

// ---- host: tensor maps ---------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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
  return fn;
}

int encode_tmap_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                     int box_cols, int box_rows) {
  auto fn = get_encode();
  if (!fn) return COSMA_ERR_CUDA;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15)) return COSMA_ERR_INVALID_ARG;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

// bf16 map of a k-blocked operand [kbt][rows][64] (64 k per 128-byte row):
// 64 x box_rows x 1 boxes, 128-byte swizzle.
static int encode_tmap_bf16_blocked(CUtensorMap* map, const void* base, int64_t rows,
                                    int64_t kbt, int box_rows) {
  auto fn = get_encode();
  if (!fn) return COSMA_ERR_CUDA;
  if (reinterpret_cast<uintptr_t>(base) & 15) return COSMA_ERR_INVALID_ARG;
  cuuint64_t dims[3] = {64, (cuuint64_t)rows, (cuuint64_t)kbt};
  cuuint64_t strides[2] = {128, (cuuint64_t)(rows * 128)};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

// f32 map for tensor stores of C: 32 x 32 boxes, 128-byte swizzle.
int encode_tmap_f32_store(CUtensorMap* map, void* base, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = get_encode();
  if (!fn) return COSMA_ERR_CUDA;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 4) & 15)) return COSMA_ERR_INVALID_ARG;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

namespace {

constexpr int BM = 128;
constexpr int BK = 64;

// Bt[j][t] = B[t][j]: k x n (ldb) -> n x k (ldt).
__global__ void transpose_bf16(const __nv_bfloat16* __restrict__ B, int64_t k, int64_t n,
                               int64_t ldb, __nv_bfloat16* __restrict__ Bt, int64_t ldt) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int64_t t0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t t = t0 + i, j = j0 + threadIdx.x;
    if (t < k && j < n) tile[i][threadIdx.x] = B[t * ldb + j];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t j = j0 + i, t = t0 + threadIdx.x;
    if (j < n && t < k) Bt[j * ldt + t] = tile[threadIdx.x][i];
  }
}

// k-blocked copy of A (m x k, lda): Ab[kb][i][0..63] = A[i][64 kb .. 64 kb + 63],
// zero beyond k.  One 16-byte chunk (8 bf16) per thread step, walking A row by
// row (contiguous reads; the writes land 128 bytes at a time in the panels).
// vec: A 16-byte aligned and lda a multiple of 8.
__global__ void block_a_bf16(const __nv_bfloat16* __restrict__ A, int64_t m, int64_t k,
                             int64_t lda, __nv_bfloat16* __restrict__ Ab, int64_t kbt, int vec) {
  const int64_t chunks = m * kbt * 8;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < chunks;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e & 7, rk = e >> 3;  // chunk q of (row i, block kb)
    const int64_t i = rk / kbt, kb = rk - i * kbt;
    const int64_t t0 = kb * 64 + q * 8;
    uint4 v;
    if (vec && t0 + 8 <= k) {
      v = *reinterpret_cast<const uint4*>(A + i * lda + t0);
    } else {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t t = t0 + 2 * j;
        const uint16_t lo = t < k ? __bfloat16_as_ushort(A[i * lda + t]) : 0;
        const uint16_t hi = t + 1 < k ? __bfloat16_as_ushort(A[i * lda + t + 1]) : 0;
        w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
      }
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    *reinterpret_cast<uint4*>(Ab + ((kb * m + i) * 64 + q * 8)) = v;
  }
}

struct TcArgs {
  Sched s;
  float* C;
  int64_t ldc;
  float* partial;
  int* status;
  long long wait_limit;
  int vec_ok;  // C rows 16-byte aligned
  float alpha, beta;  // C = alpha A B + beta C (C read only when beta != 0)
  int c_tma;          // C written by tensor stores (pk == 1, beta == 0, aligned rows)
  int a_blocked;      // A read from its k-blocked copy [kbt][m][64] (3-D map)
};

template <int BN, int STAGES>
struct Layout {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  // epilogue staging: per epilogue warp two 32 x 32 f32 boxes (128-byte swizzle)
  static constexpr int EPI_OFF = STAGES * STAGE_BYTES;
  static constexpr int EPI_BYTES = 4 * 2 * 4096;
  static constexpr int BAR_OFF = EPI_OFF + EPI_BYTES;
  static constexpr int NBARS = 2 * STAGES + 5;  // full, empty, tfull[2], tempty[2], drain
  static constexpr int TOTAL = BAR_OFF + NBARS * 8 + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};

__device__ __forceinline__ void store_row32(float* dst, int64_t col0, int64_t n, const uint32_t (&r)[32],
                                            bool vec, float alpha = 1.f, float beta = 0.f) {
  if (alpha != 1.f || beta != 0.f) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (col0 + j >= n) continue;
      float v = alpha * __uint_as_float(r[j]);
      if (beta != 0.f) v = fmaf(beta, dst[j], v);
      dst[j] = v;
    }
    return;
  }
  if (vec && col0 + 32 <= n) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      d4[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                          __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (col0 + j < n) dst[j] = __uint_as_float(r[j]);
  }
}

template <int BN, int STAGES, bool A_MN, bool B_MN>
__global__ void __launch_bounds__(192, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, TcArgs a) {
  using L = Layout<BN, STAGES>;
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
  if (warp == 1) tc::tmem_alloc(tslot, 2 * BN);
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
      // the next unit is decoded while this one's first stage is in flight
      Unit nxt = nunits > 0 ? unit_of_cta(a.s, cta, 0) : Unit{};
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        const Unit u = nxt;
        bool ok = true;
        for (int64_t kb = u.kb0; kb < u.kb1; ++kb) {
          if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&full[stage], L::STAGE_BYTES);
          uint8_t* sa = smem + stage * L::STAGE_BYTES;
          if constexpr (A_MN) {
#pragma unroll
            for (int j = 0; j < BM / 64; ++j)  // box j: rows j*64.. of the tile, k rows kb*64..
              tc::tma_load_2d(sa + j * (64 * BK * 2), &tmA, &full[stage],
                              (int32_t)(u.tile_row * BM + j * 64), (int32_t)(kb * BK));
          } else if (a.a_blocked) {
            tc::tma_load_3d(sa, &tmA, &full[stage], 0, (int32_t)(u.tile_row * BM), (int32_t)kb);
          } else {
            tc::tma_load_2d(sa, &tmA, &full[stage], (int32_t)(kb * BK),
                            (int32_t)(u.tile_row * BM));
          }
          if constexpr (B_MN) {
#pragma unroll
            for (int j = 0; j < BN / 64; ++j)  // box j: columns j*64.., k rows kb*64..
              tc::tma_load_2d(sa + L::A_BYTES + j * (64 * BK * 2), &tmB, &full[stage],
                              (int32_t)(u.tile_col * BN + j * 64), (int32_t)(kb * BK));
          } else {
            tc::tma_load_2d(sa + L::A_BYTES, &tmB, &full[stage], (int32_t)(kb * BK),
                            (int32_t)(u.tile_col * BN));
          }
          armed |= 1u << stage;
          armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
          if (++stage == STAGES) { stage = 0; ph ^= 1; }
          if (kb == u.kb0 && ui + 1 < nunits) nxt = unit_of_cta(a.s, cta, ui + 1);
        }
        if (!ok) break;
        if (u.kb0 >= u.kb1 && ui + 1 < nunits) nxt = unit_of_cta(a.s, cta, ui + 1);
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
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN) | (A_MN ? (1u << 15) : 0u) |
                                 (B_MN ? (1u << 16) : 0u);
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[2] = {0, 0};
      for (int64_t ui = 0; ui < nunits && !*abort_flag; ++ui) {
        int64_t kb0, kb1;
        unit_k_range(a.s, cta, ui, kb0, kb1);
        if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) break;
        tc::tc_fence_after();
        const uint32_t d = tmem_base + acc * BN;
        bool ok = true;
        for (int64_t kb = kb0; kb < kb1; ++kb) {
          if (!tc::mbar_wait(&full[stage], ph, w)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
          const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            // B MN-major: 16 k rows of 128 bytes per step; boxes 64 x BK apart
            const uint64_t db = B_MN ? tc::smem_desc_mn_sw128(sb + kk * 16 * 128, 64 * BK * 2, 1024)
                                     : tc::smem_desc_sw128(sb + kk * 32);
            const uint64_t da = A_MN ? tc::smem_desc_mn_sw128(sa + kk * 16 * 128, 64 * BK * 2, 1024)
                                     : tc::smem_desc_sw128(sa + kk * 32);
            tc::mma_bf16(d, da, db, idesc, (kb > kb0 || kk > 0) ? 1u : 0u);
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == STAGES) { stage = 0; ph ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit(&tfull[acc]);
        aph[acc] ^= 1;
        acc ^= 1;
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
    uint8_t* stage_c = smem + L::EPI_OFF + q * 8192;  // this warp's two staging boxes
    uint32_t stores = 0;                               // tensor stores committed so far
    const int64_t n4 = a.s.n & ~(int64_t)3;            // columns the C map covers
    if (warp == 2 && lane == 0 && a.c_tma) tc::prefetch_tmap(&tmC);
    for (int64_t ui = 0; ui < nunits; ++ui) {
      const Unit u = unit_of_cta(a.s, cta, ui);
      if (!tc::mbar_wait(&tfull[acc], tph[acc], w)) break;
      tc::tc_fence_after();
      const int64_t row0 = u.tile_row * BM + q * 32;
      const int64_t row = row0 + lane;
      float* dst_row = nullptr;
      if (row < a.s.m) {
        dst_row = a.s.pk > 1 ? a.partial + (int64_t)u.ks * a.s.m * a.s.n + row * a.s.n
                             : a.C + row * a.ldc;
      }
      const bool vec = a.s.pk > 1 ? ((a.s.n & 3) == 0) : (a.vec_ok != 0);
      // One 32-column chunk of the accumulator, already in registers.
      auto chunk = [&](const uint32_t (&r)[32], int c) {
        const int64_t col0 = u.tile_col * BN + c;
        if (a.c_tma) {
          // Columns below n4: this warp's 32 rows -> one 32 x 32 box in shared memory
          // (16-byte chunk j of row l at chunk j ^ (l % 8): the 128-byte swizzle), then
          // one tensor store clipped at m and n4 (a store clips in whole 16-byte units);
          // columns n4..n-1 are written by the lanes.
          if (row0 >= a.s.m || col0 >= a.s.n) return;
          if (col0 < n4) {
            uint8_t* box = stage_c + (stores & 1) * 4096;
            if (lane == 0) tc::bulk_wait_read<1>();  // the box's previous store has read it
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float4 v = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                     __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
              if (a.alpha != 1.f) { v.x *= a.alpha; v.y *= a.alpha; v.z *= a.alpha; v.w *= a.alpha; }
              *reinterpret_cast<float4*>(box + lane * 128 + ((j ^ (lane & 7)) * 16)) = v;
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              tc::tma_store_2d(&tmC, box, (int32_t)col0, (int32_t)row0);
              tc::bulk_commit();
            }
            ++stores;
          }
          if (dst_row && col0 + 32 > n4) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col0 + j >= n4 && col0 + j < a.s.n) dst_row[col0 + j] = a.alpha * __uint_as_float(r[j]);
          }
          return;
        }
        if (dst_row && col0 < a.s.n) {
          if (a.s.pk > 1) store_row32(dst_row + col0, col0, a.s.n, r, vec);
          else store_row32(dst_row + col0, col0, a.s.n, r, vec, a.alpha, a.beta);
        }
      };
      // Two register sets: the next chunk's tensor-memory load is in flight while
      // the current one is written out.
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + acc * BN;
      uint32_t ra[32], rb[32];
      tc::tmem_ld_32x32(tbase, ra);
      tc::tmem_wait_ld_r32(ra);
#pragma unroll 1
      for (int c = 0; c < BN; c += 64) {
        tc::tmem_ld_32x32(tbase + c + 32, rb);
        chunk(ra, c);
        tc::tmem_wait_ld_r32(rb);
        if (c + 64 < BN) tc::tmem_ld_32x32(tbase + c + 64, ra);
        chunk(rb, c + 32);
        if (c + 64 < BN) tc::tmem_wait_ld_r32(ra);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[acc]);
      tph[acc] ^= 1;
      acc ^= 1;
    }
    if (lane == 0) tc::bulk_wait_all();  // stores done before shared memory goes away
    __syncwarp();
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, 2 * BN);
  }
}

template <int BN, int STAGES, bool A_MN, bool B_MN>
int launch_kernel(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tcm,
                  const TcArgs& args, cudaStream_t st) {
  using L = Layout<BN, STAGES>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES, A_MN, B_MN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC);
  });
  if (attr != cudaSuccess) return (int)attr;
  prof_mark(st, true);
  tc_gemm_kernel<BN, STAGES, A_MN, B_MN><<<args.s.ctas, 192, L::ALLOC, st>>>(ta, tb, tcm, args);
  prof_mark(st, false);
  count_launch();
  return (int)cudaGetLastError();
}

inline int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

}  // namespace

bool tc_b_direct(const void* B, int64_t ldb);

// Bytes of the operand copies launch_tc_bf16 makes (see there).
struct TcCopies {
  bool a_mn, b_mn;      // operands multiplied MN-major
  bool pack_a, copy_b;  // A copied to the workspace; B copied (transposed or packed)
  bool b_transpose;     // the B copy is a transpose (else a packed copy of B^T)
  bool block_a;         // A copied k-blocked: its rows are too far apart for one box
};

// Row pitch (bytes) from which a K-major A is read through its k-blocked copy: a
// 128-row box then touches 128 pages of memory (16 at 256 KB), and the tensor
// cores wait on translation -- 0.66 of peak at k = 2^20 (rows 2 MB apart).
constexpr int64_t kBlockARowBytes = 256 << 10;

static TcCopies tc_copies(const void* A, int64_t lda, int trans_a, const void* B, int64_t ldb,
                          int trans_b, int64_t k) {
  TcCopies c;
  const bool a_ok = A && (reinterpret_cast<uintptr_t>(A) & 15) == 0 && ((lda * 2) & 15) == 0;
  const bool b_ok = B && (reinterpret_cast<uintptr_t>(B) & 15) == 0 && ((ldb * 2) & 15) == 0;
  c.a_mn = trans_a != 0;
  c.block_a = !trans_a && lda * 2 >= kBlockARowBytes && k >= 8 * BK;
  c.pack_a = !a_ok && !c.block_a;
  c.b_mn = !trans_b && b_ok;
  c.copy_b = !c.b_mn && !(trans_b && b_ok);
  c.b_transpose = !trans_b;
  return c;
}

int launch_tc_bf16(const GemmArgs& g, const Sched& s, const cosma_plan& p, void* ws,
                   long long ws_bytes, int* status, long long wait_limit, cudaStream_t st) {
  const int64_t kp = round_up(g.k, 8), mp = round_up(g.m, 8);
  const TcCopies cp = tc_copies(g.A, g.lda, g.trans_a, g.B, g.ldb, g.trans_b, g.k);
  uint8_t* w = static_cast<uint8_t*>(ws);
  long long off = 0;
  float* partial = nullptr;
  if (p.pk > 1) {
    partial = reinterpret_cast<float*>(w + off);
    off += round_up((long long)p.pk * g.m * g.n * 4, 256);
  }
  // B operand: in place (MN-major when stored k x n, K-major when stored n x k),
  // else a K-major n x kp copy (a transpose of k x n, or a pitch-padded copy of n x k).
  const __nv_bfloat16* Buse = static_cast<const __nv_bfloat16*>(g.B);
  int64_t ldb = g.ldb;
  if (cp.copy_b) {
    __nv_bfloat16* Bt = reinterpret_cast<__nv_bfloat16*>(w + off);
    off += round_up(g.n * kp * 2, 256);
    if (off > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
    if (cp.b_transpose) {
      dim3 grid((unsigned)((g.n + 31) / 32), (unsigned)((g.k + 31) / 32));
      if (grid.y > 65535) return COSMA_ERR_UNSUPPORTED;
      transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(static_cast<const __nv_bfloat16*>(g.B), g.k,
                                                   g.n, g.ldb, Bt, kp);
      count_launch();
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return (int)e;
    } else if (cudaMemcpy2DAsync(Bt, kp * 2, g.B, g.ldb * 2, g.k * 2, g.n,
                                 cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      return (int)cudaGetLastError();
    }
    Buse = Bt;
    ldb = kp;
  }
  // A operand: in place, else a copy with a 16-byte pitch (m x kp, or k x mp when
  // stored transposed).
  const __nv_bfloat16* Ause = static_cast<const __nv_bfloat16*>(g.A);
  int64_t lda = g.lda;
  if (cp.pack_a) {
    __nv_bfloat16* Ap = reinterpret_cast<__nv_bfloat16*>(w + off);
    const int64_t rows = cp.a_mn ? g.k : g.m, cols = cp.a_mn ? g.m : g.k;
    const int64_t pitch = cp.a_mn ? mp : kp;
    off += round_up(rows * pitch * 2, 256);
    if (off > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
    if (cudaMemcpy2DAsync(Ap, pitch * 2, g.A, g.lda * 2, cols * 2, rows, cudaMemcpyDeviceToDevice,
                          st) != cudaSuccess)
      return (int)cudaGetLastError();
    Ause = Ap;
    lda = pitch;
  }
  const int64_t kbt = (g.k + BK - 1) / BK;
  if (cp.block_a) {
    __nv_bfloat16* Ab = reinterpret_cast<__nv_bfloat16*>(w + off);
    off += round_up(kbt * g.m * BK * 2, 256);
    if (off > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
    int64_t blocks = (g.m * kbt * 8 + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    const int vec = ((reinterpret_cast<uintptr_t>(g.A) & 15) == 0 && (g.lda & 7) == 0) ? 1 : 0;
    block_a_bf16<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(g.A), g.m,
                                                    g.k, g.lda, Ab, kbt, vec);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    Ause = Ab;
  }
  if (off > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
  CUtensorMap ta, tb;
  int rc = cp.block_a ? encode_tmap_bf16_blocked(&ta, Ause, g.m, kbt, BM)
           : cp.a_mn  ? encode_tmap_bf16(&ta, Ause, g.k, g.m, lda, 64, BK)   // k rows of m
                      : encode_tmap_bf16(&ta, Ause, g.m, g.k, lda, BK, BM);  // m rows of k
  if (rc != COSMA_OK) return rc;
  rc = cp.b_mn ? encode_tmap_bf16(&tb, Buse, g.k, g.n, ldb, 64, BK)        // k rows of n
               : encode_tmap_bf16(&tb, Buse, g.n, g.k, ldb, BK, p.tile_n);  // n rows of k
  if (rc != COSMA_OK) return rc;
  TcArgs args;
  args.s = s;
  args.C = static_cast<float*>(g.C);
  args.ldc = g.ldc;
  args.partial = partial;
  args.status = status;
  args.wait_limit = wait_limit;
  args.vec_ok = ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0 && (g.ldc & 3) == 0) ? 1 : 0;
  args.a_blocked = cp.block_a ? 1 : 0;
  args.alpha = (float)g.alpha;
  args.beta = (float)g.beta;
  // C by tensor stores when it is written directly with 16-byte aligned rows and
  // not read (beta == 0); the map is n rounded down to 4 wide.
  CUtensorMap tcm;
  memset(&tcm, 0, sizeof(tcm));
  args.c_tma = 0;
  if (p.pk == 1 && g.beta == 0.0 && g.n >= 4 && args.vec_ok) {
    rc = encode_tmap_f32_store(&tcm, g.C, g.m, g.n & ~(int64_t)3, g.ldc);
    if (rc != COSMA_OK) return rc;
    args.c_tma = 1;
  }
  const bool wide = p.tile_n == 256;
  int err;
  if (cp.a_mn && cp.b_mn)
    err = wide ? launch_kernel<256, 4, true, true>(ta, tb, tcm, args, st)
               : launch_kernel<128, 6, true, true>(ta, tb, tcm, args, st);
  else if (cp.a_mn)
    err = wide ? launch_kernel<256, 4, true, false>(ta, tb, tcm, args, st)
               : launch_kernel<128, 6, true, false>(ta, tb, tcm, args, st);
  else if (cp.b_mn)
    err = wide ? launch_kernel<256, 4, false, true>(ta, tb, tcm, args, st)
               : launch_kernel<128, 6, false, true>(ta, tb, tcm, args, st);
  else
    err = wide ? launch_kernel<256, 4, false, false>(ta, tb, tcm, args, st)
               : launch_kernel<128, 6, false, false>(ta, tb, tcm, args, st);
  if (err) return err;
  if (p.pk > 1) return launch_reduce(COSMA_F32, g, p.pk, partial, st);
  return 0;
}

// f32 parts [2][kbt][rows][32]: dims (32, rows, kbt, 2), 32 x box_rows x 1 x 1 boxes,
// 128-byte swizzle.
int encode_tmap_f32_parts(CUtensorMap* map, const float* base, int64_t rows, int64_t kbt,
                          int box_rows) {
  auto fn = get_encode();
  if (!fn) return COSMA_ERR_CUDA;
  cuuint64_t dims[4] = {32, (cuuint64_t)rows, (cuuint64_t)kbt, 2};
  cuuint64_t strides[3] = {128, (cuuint64_t)(rows * 128), (cuuint64_t)(kbt * rows * 128)};
  cuuint32_t box[4] = {32, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

bool tc_b_direct(const void* B, int64_t ldb) {
  return (reinterpret_cast<uintptr_t>(B) & 15) == 0 && ((ldb * 2) & 15) == 0;
}

long long tc_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_plan& p, const void* A,
                             int64_t lda, int trans_a, const void* B, int64_t ldb, int trans_b) {
  const int64_t kp = round_up(k, 8), mp = round_up(m, 8);
  const TcCopies cp = tc_copies(A, lda, trans_a, B, ldb, trans_b, k);
  long long b = 0;
  if (p.pk > 1) b += round_up((long long)p.pk * m * n * 4, 256);
  if (cp.copy_b) b += round_up(n * kp * 2, 256);
  if (cp.pack_a) b += round_up((cp.a_mn ? k * mp : m * kp) * 2, 256);
  if (cp.block_a) b += round_up((k + BK - 1) / BK * m * BK * 2, 256);
  return b;
}

}  // namespace cosma

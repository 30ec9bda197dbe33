// K-GROUPED: many independent products C_i = A_i B_i in one persistent launch.
//
// Batching pattern (not in the paper).  The host builds, once per distinct
// group, a device table: per problem its TMA tensor maps and sizes, and a
// static assignment of all (problem, tile) work units to CTAs -- units sorted
// by cost (k blocks) and handed to the least-loaded CTA (longest processing
// time first; each CTA then runs its units cheapest first), so no atomics or
// device queue are needed.  Each CTA then runs
// the C-stationary schedule of Listing 1 on its units exactly as the
// single-product kernels do: bf16 on tcgen05 (TMA ring, TMEM accumulators),
// f32 on the FMA pipes.  B_i (k x n) is first transposed into the workspace
// by one grouped prep launch so both MMA operands are K-major.
//
// The table is cached (by the problems' contents, the tile and the workspace
// address): after one eager call the same call can be captured in a CUDA
// graph, because a cache hit launches kernels only (no allocation, no host
// copy).  Up to kCacheSlots groups stay cached per device; a table that a
// capture recorded is never overwritten: when its slot is reused the table
// moves to a retired list, freed at cosma_finalize, so the graph stays valid.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <mutex>
#include <queue>
#include <vector>

#include "simt_f32.cuh"
#include "simt_tile.cuh"
#include "tc_common.cuh"

namespace cosma {

namespace {

constexpr int GBM = 128, GBK = 64;
// Problems whose A and B tensor maps a CTA remembers having acquired (a shared-memory
// bitmap): each is acquired once per CTA; problems beyond it on every change.
constexpr int kAcqWords = 128;
constexpr int kCacheSlots = 8;

struct alignas(128) GMap {
  CUtensorMap ta;
  CUtensorMap tb;
  CUtensorMap tc;  // f32 C, 32 x 32 boxes (stores), when c_tma
};

struct GMeta {
  int64_t m, n, k;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  __nv_bfloat16* Bt;  // bf16: B transposed (n x kp)
  int64_t ldt;
  __nv_bfloat16* Ap;  // bf16: A copied with a 16-byte row pitch when its own is not
  int64_t ldap;
  int vec_ok;
  int f32_async;  // f32: A, B 16-byte aligned with pitches multiple of 4 floats
  int b_mn;       // bf16: B loaded as it is (MN-major operand), no transposed copy
  int c_tma;      // bf16: C written by tensor stores (16-byte aligned rows)
};

struct GUnit {
  int p, tile_row, tile_col;
  int kbf;  // bf16: k blocks << 1 | b_mn of the problem, so the producer and the
            // MMA issuer start a unit from this record alone
};

struct Table {
  unsigned long long key = 0;
  int count = 0, dtype = -1, tile_n = 0, ctas = 0;
  void* dev = nullptr;  // device copy
  size_t bytes = 0;
  // device views
  const GMap* maps = nullptr;
  const GMeta* meta = nullptr;
  const GUnit* units = nullptr;
  const int* cta_off = nullptr;
  const int64_t* tprefix = nullptr;  // transpose-tile prefix, count + 1
  const int64_t* aprefix = nullptr;  // A-copy-tile prefix, count + 1
  int64_t ttiles = 0;
  int64_t atiles = 0;
  int64_t nunits = 0;
  bool captured = false;  // recorded in a captured graph
};

std::mutex g_tab_mu;
Table g_cache[16][kCacheSlots];
int g_next[16];
std::vector<void*> g_retired[16];  // tables of captured graphs, freed at finalize

inline int64_t rup(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

unsigned long long mix(unsigned long long h, unsigned long long v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

// ---- kernels -------------------------------------------------------------------

__device__ __forceinline__ int find_problem(const int64_t* prefix, int count, int64_t x) {
  int lo = 0, hi = count;  // prefix[lo] <= x < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Transposes every B_i (k x n) into Bt_i (n x kp) and copies each A_i whose
// row pitch is not a multiple of 16 bytes into Ap_i (m x kp).  64 x 64 tiles,
// 256 threads: each warp moves rows of 64 elements as 32 pairs (4 bytes per
// lane) when the pitch allows, single elements otherwise.
constexpr int PT = 64;

__global__ void __launch_bounds__(256)
grouped_prep_kernel(const GMeta* __restrict__ meta, const int64_t* __restrict__ tprefix,
                    const int64_t* __restrict__ aprefix, int count, int64_t ttiles,
                    int64_t atiles) {
  __shared__ __nv_bfloat16 tile[PT][PT + 2];
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
  for (int64_t x = blockIdx.x; x < ttiles + atiles; x += gridDim.x) {
    if (x < ttiles) {
      const int p = find_problem(tprefix, count, x);
      const GMeta& g = meta[p];
      const int64_t local = x - tprefix[p];
      const int64_t tiles_j = (g.n + PT - 1) / PT;
      const int64_t t0 = (local / tiles_j) * PT, j0 = (local % tiles_j) * PT;
      const __nv_bfloat16* B = static_cast<const __nv_bfloat16*>(g.B);
      const bool pairs_in = ((g.ldb & 1) == 0) && ((reinterpret_cast<uintptr_t>(B) & 3) == 0);
      __syncthreads();
      for (int r = wrp; r < PT; r += 8) {  // rows t of B, columns j
        const int64_t t = t0 + r, j = j0 + 2 * lane;
        if (t >= g.k) continue;
        if (pairs_in && j + 1 < g.n) {
          const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(B + t * g.ldb + j);
          tile[r][2 * lane] = v.x;
          tile[r][2 * lane + 1] = v.y;
        } else {
          if (j < g.n) tile[r][2 * lane] = B[t * g.ldb + j];
          if (j + 1 < g.n) tile[r][2 * lane + 1] = B[t * g.ldb + j + 1];
        }
      }
      __syncthreads();
      for (int r = wrp; r < PT; r += 8) {  // rows j of Bt, columns t (ldt is even)
        const int64_t j = j0 + r, t = t0 + 2 * lane;
        if (j >= g.n) continue;
        if (t + 1 < g.k) {
          __nv_bfloat162 v;
          v.x = tile[2 * lane][r];
          v.y = tile[2 * lane + 1][r];
          *reinterpret_cast<__nv_bfloat162*>(g.Bt + j * g.ldt + t) = v;
        } else if (t < g.k) {
          g.Bt[j * g.ldt + t] = tile[2 * lane][r];
        }
      }
    } else {
      const int64_t y = x - ttiles;
      const int p = find_problem(aprefix, count, y);
      const GMeta& g = meta[p];
      const int64_t local = y - aprefix[p];
      const int64_t tiles_t = (g.k + PT - 1) / PT;
      const int64_t r0 = (local / tiles_t) * PT, t0 = (local % tiles_t) * PT;
      const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(g.A);
      for (int i = wrp; i < PT; i += 8) {
        const int64_t r = r0 + i;
        if (r >= g.m) continue;
        for (int c = lane; c < PT; c += 32) {
          const int64_t t = t0 + c;
          if (t < g.k) g.Ap[r * g.ldap + t] = A[r * g.lda + t];
        }
      }
    }
  }
}

struct GArgs {
  const GMap* maps;
  const GMeta* meta;
  const GUnit* units;
  const int* cta_off;
  int* status;
  long long wait_limit;
};

template <int BN, int STAGES>
struct GLayout {
  static constexpr int A_BYTES = GBM * GBK * 2;
  static constexpr int B_BYTES = BN * GBK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  // epilogue staging: per epilogue warp two 32 x 32 f32 boxes (128-byte swizzle)
  static constexpr int EPI_OFF = STAGES * STAGE_BYTES;
  static constexpr int EPI_BYTES = 4 * 2 * 4096;
  static constexpr int BAR_OFF = EPI_OFF + EPI_BYTES;
  static constexpr int NBARS = 2 * STAGES + 5;
  static constexpr int ACQ_OFF = BAR_OFF + NBARS * 8 + 16;  // tensor maps acquired
  static constexpr int TOTAL = ACQ_OFF + 4 * kAcqWords;
  static constexpr int ALLOC = TOTAL + 1024;
};

__device__ __forceinline__ void acquire_tmap(const CUtensorMap* m);

// The producer's acquire of problem p's operand maps before its first copies from
// them: once per CTA for the problems the bitmap covers.
__device__ __forceinline__ void acquire_maps_once(uint32_t* acq, int p, const CUtensorMap* ta,
                                                  const CUtensorMap* tb) {
  const bool tracked = p < kAcqWords * 32;
  if (tracked && ((acq[p >> 5] >> (p & 31)) & 1u)) return;
  acquire_tmap(ta);
  acquire_tmap(tb);
  if (tracked) acq[p >> 5] |= 1u << (p & 31);
}

__device__ __forceinline__ void acquire_tmap(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                   reinterpret_cast<uint64_t>(m))
               : "memory");
}

// Epilogue warps of the grouped tensor-core kernels, one per tensor-memory lane
// quadrant q: for each unit, wait for its accumulator, write this CTA's 32 rows
// of the C tile -- tensor stores through the warp's two 4 KB staging boxes
// (stage_c) where C allows them, else the lanes' own stores -- and report the
// accumulator free with free_acc(acc).  TM: rows of a unit's tile; row_off: this
// CTA's first row in it.
template <int BN, int TM, class FreeAcc>
__device__ __forceinline__ void grouped_epilogue(const GArgs& a, int u0, int u1,
                                                 uint32_t tmem_base, uint64_t* tfull,
                                                 uint8_t* stage_c, int64_t row_off,
                                                 const tc::WaitCtx& w, int q, int lane,
                                                 FreeAcc free_acc) {
  uint32_t acc = 0;
  uint32_t tph[2] = {0, 0};
  uint32_t stores = 0;  // tensor stores committed so far
  for (int ui = u0; ui < u1; ++ui) {
    const GUnit u = a.units[ui];
    // the problem's fields are loaded before the wait, so their latency hides in it
    struct {
      int64_t m, n, ldc;
      float* C;
      int c_tma, vec_ok;
    } g;
    {
      const GMeta& gm = a.meta[u.p];
      g.m = gm.m;
      g.n = gm.n;
      g.ldc = gm.ldc;
      g.C = static_cast<float*>(gm.C);
      g.c_tma = gm.c_tma;
      g.vec_ok = gm.vec_ok;
    }
    if (!tc::mbar_wait(&tfull[acc], tph[acc], w)) break;
    tc::tc_fence_after();
    const int64_t row0 = (int64_t)u.tile_row * TM + row_off + q * 32;
    const int64_t row = row0 + lane;
    float* dst_row = row < g.m ? g.C + row * g.ldc : nullptr;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      uint32_t r[32];
      tc::tmem_ld_32x32(tmem_base + ((uint32_t)(q * 32) << 16) + acc * BN + c, r);
      tc::tmem_wait_ld_r32(r);  // r is read only after the wait
      const int64_t col0 = (int64_t)u.tile_col * BN + c;
      if (g.c_tma) {
        // Columns below n4 = n rounded down to 4: rows of this warp -> one 32 x 32
        // box in shared memory (16-byte chunk j of row l at chunk j ^ (l % 8): the
        // 128-byte swizzle), then one tensor store, which clips at m and n4 (the C
        // map is n4 wide: a store clips in whole 16-byte units).  Columns n4..n-1
        // are written by the lanes themselves.
        if (row0 >= g.m || col0 >= g.n) continue;
        const int64_t n4 = g.n & ~(int64_t)3;
        if (col0 < n4) {
          uint8_t* box = stage_c + (stores & 1) * 4096;
          if (lane == 0) tc::bulk_wait_read<1>();  // the box's previous store has read it
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float4*>(box + lane * 128 + ((j ^ (lane & 7)) * 16)) =
                make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                            __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tc::tma_store_2d(&a.maps[u.p].tc, box, (int32_t)col0, (int32_t)row0);
            tc::bulk_commit();
          }
          ++stores;
        }
        if (dst_row && col0 + 32 > n4) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j >= n4 && col0 + j < g.n) dst_row[col0 + j] = __uint_as_float(r[j]);
        }
        continue;
      }
      if (dst_row && col0 < g.n) {
        float* dst = dst_row + col0;
        if (g.vec_ok && col0 + 32 <= g.n) {
          float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            d4[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j < g.n) dst[j] = __uint_as_float(r[j]);
        }
      }
    }
    tc::tc_fence_before();
    __syncwarp();
    if (lane == 0) free_acc(acc);
    tph[acc] ^= 1;
    acc ^= 1;
  }
  if (lane == 0) tc::bulk_wait_all();  // stores done before shared memory goes away
  __syncwarp();
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(192, 1) grouped_tc_kernel(GArgs a) {
  using L = GLayout<BN, STAGES>;
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
  uint32_t* acq = reinterpret_cast<uint32_t*>(smem + L::ACQ_OFF);

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
    for (int i = 0; i < kAcqWords; ++i) acq[i] = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(tslot, 2 * BN);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const tc::WaitCtx w{a.wait_limit, a.status, abort_flag};
  const int u0 = a.cta_off[blockIdx.x], u1 = a.cta_off[blockIdx.x + 1];

  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0, armed = 0, armed_ph = 0;
      int last_p = -1;
      GUnit nu = u0 < u1 ? a.units[u0] : GUnit{};
      for (int ui = u0; ui < u1 && !*abort_flag; ++ui) {
        const GUnit u = nu;
        if (ui + 1 < u1) nu = a.units[ui + 1];  // in flight while this unit's loads issue
        const CUtensorMap* ta = &a.maps[u.p].ta;
        const CUtensorMap* tb = &a.maps[u.p].tb;
        if (u.p != last_p) {
          acquire_maps_once(acq, u.p, ta, tb);
          last_p = u.p;
        }
        const int64_t kbt = u.kbf >> 1;
        const bool bmn = (u.kbf & 1) != 0;
        bool ok = true;
        for (int64_t kb = 0; kb < kbt; ++kb) {
          if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&full[stage], L::STAGE_BYTES);
          uint8_t* sa = smem + stage * L::STAGE_BYTES;
          tc::tma_load_2d(sa, ta, &full[stage], (int32_t)(kb * GBK), u.tile_row * GBM);
          if (bmn) {
#pragma unroll
            for (int j = 0; j < BN / 64; ++j)  // box j: columns j*64.., k rows kb*64..
              tc::tma_load_2d(sa + L::A_BYTES + j * (64 * GBK * 2), tb, &full[stage],
                              u.tile_col * BN + j * 64, (int32_t)(kb * GBK));
          } else {
            tc::tma_load_2d(sa + L::A_BYTES, tb, &full[stage], (int32_t)(kb * GBK),
                            u.tile_col * BN);
          }
          armed |= 1u << stage;
          armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
          if (++stage == STAGES) { stage = 0; ph ^= 1; }
        }
        if (!ok) break;
      }
      if (*abort_flag) {
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
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[2] = {0, 0};
      GUnit nu = u0 < u1 ? a.units[u0] : GUnit{};
      for (int ui = u0; ui < u1 && !*abort_flag; ++ui) {
        const GUnit u = nu;
        if (ui + 1 < u1) nu = a.units[ui + 1];
        const int64_t kbt = u.kbf >> 1;
        const bool bmn = (u.kbf & 1) != 0;
        const uint32_t idesc =
            bmn ? tc::idesc_bf16_f32_bmn(GBM, BN) : tc::idesc_bf16_f32(GBM, BN);
        if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) break;
        tc::tc_fence_after();
        const uint32_t d = tmem_base + acc * BN;
        bool ok = true;
        for (int64_t kb = 0; kb < kbt; ++kb) {
          if (!tc::mbar_wait(&full[stage], ph, w)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
          const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < GBK / 16; ++kk) {
            const uint64_t db = bmn ? tc::smem_desc_mn_sw128(sb + kk * 16 * 128, 64 * GBK * 2, 1024)
                                    : tc::smem_desc_sw128(sb + kk * 32);
            tc::mma_bf16(d, tc::smem_desc_sw128(sa + kk * 32), db, idesc,
                         (kb > 0 || kk > 0) ? 1u : 0u);
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == STAGES) { stage = 0; ph ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit(&tfull[acc]);
        aph[acc] ^= 1;
        acc ^= 1;
      }
      tc::mma_commit(drain);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  } else {
    const int q = warp & 3;
    grouped_epilogue<BN, GBM>(a, u0, u1, tmem_base, tfull, smem + L::EPI_OFF + q * 8192, 0, w,
                              q, lane, [&](uint32_t b) { tc::mbar_arrive(&tempty[b]); });
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, 2 * BN);
  }
}

// ---- CTA-pair variant (bf16, grouped_tile 512) --------------------------------------
//
// 256 x 256 C tiles on clusters of two CTAs (tcgen05.mma.cta_group::2, M = 256,
// N = 256): each CTA loads its own 128 rows of A and its own 128 of the tile's 256
// columns of B (no multicast), the even CTA issues the MMAs and commits to the
// barriers of both, and each CTA drains its own 128 x 256 accumulator.  Per SM a
// 64-deep k block moves 32 KB of operands for 128 x 256 x 64 products instead of
// 48 KB, so the same shared memory keeps six k blocks in flight instead of four.

constexpr int GPS = 6;  // ring stages of the pair kernel
struct GPairLayout {
  static constexpr int A_BYTES = GBM * GBK * 2;      // own 128 rows
  static constexpr int B_BYTES = 128 * GBK * 2;      // own 128 columns
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int EPI_OFF = GPS * STAGE_BYTES;
  static constexpr int EPI_BYTES = 4 * 2 * 4096;
  static constexpr int BAR_OFF = EPI_OFF + EPI_BYTES;
  // full, empty, tfull, tempty, drain, peer-count exchange
  static constexpr int NBARS = 2 * GPS + 2 * 2 + 2;
  static constexpr int ACQ_OFF = BAR_OFF + NBARS * 8 + 16;  // tensor maps acquired
  static constexpr int TOTAL = ACQ_OFF + 4 * kAcqWords;
  static constexpr int ALLOC = TOTAL + 1024;
};

// One box of a 2-D bf16 map into this CTA's shared memory; its bytes are counted on
// the barrier at bar_cluster (the leader CTA's).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];\n" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}

__global__ void __launch_bounds__(192, 1) grouped_pair_kernel(GArgs a) {
  using L = GPairLayout;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + GPS;
  uint64_t* tfull = empty + GPS;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint64_t* xchg = drain + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(xchg + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  uint32_t* peer_issued = tslot + 2;
  uint32_t* acq = reinterpret_cast<uint32_t*>(smem + L::ACQ_OFF);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = tc::cluster_ctarank();
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GPS; ++s) {
      tc::mbar_init(&full[s], 1);   // leader: its producer's arrival + both CTAs' bytes
      tc::mbar_init(&empty[s], 1);  // the leader's commit, multicast to both CTAs
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 8);  // leader: the 4 epilogue warps of each CTA
    }
    tc::mbar_init(drain, 1);
    tc::mbar_init(xchg, 1);  // leader: the odd CTA's count of issued stages
    *abort_flag = 0;
    *peer_issued = 0;
    for (int i = 0; i < kAcqWords; ++i) acq[i] = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc_pair(tslot, 512);
  tc::tc_fence_before();
  tc::cluster_sync();  // barriers of both CTAs initialised, tensor memory allocated
  tc::tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const tc::WaitCtx w{a.wait_limit, a.status, abort_flag};
  const int pair = blockIdx.x >> 1;
  const int u0 = a.cta_off[pair], u1 = a.cta_off[pair + 1];

  if (warp == 0) {
    if (tc::elect_one()) {
      int stage = 0;
      uint32_t ph = 0;
      uint32_t issued = 0;  // stages whose copies this CTA issued
      uint32_t full_cl[GPS];
#pragma unroll
      for (int s = 0; s < GPS; ++s) full_cl[s] = tc::mapa_shared(&full[s], 0);
      int last_p = -1;
      GUnit nu = u0 < u1 ? a.units[u0] : GUnit{};
      for (int ui = u0; ui < u1 && !*abort_flag; ++ui) {
        const GUnit u = nu;
        if (ui + 1 < u1) nu = a.units[ui + 1];  // in flight while this unit's loads issue
        const CUtensorMap* ta = &a.maps[u.p].ta;
        const CUtensorMap* tb = &a.maps[u.p].tb;
        if (u.p != last_p) {
          acquire_maps_once(acq, u.p, ta, tb);
          last_p = u.p;
        }
        const int64_t kbt = u.kbf >> 1;
        const bool bmn = (u.kbf & 1) != 0;
        const int32_t arow = u.tile_row * 256 + (int32_t)rank * 128;
        const int32_t bcol = u.tile_col * 256 + (int32_t)rank * 128;
        bool ok = true;
        for (int64_t kb = 0; kb < kbt; ++kb) {
          if (!tc::mbar_wait(&empty[stage], ph ^ 1, w)) { ok = false; break; }
          if (leader) tc::mbar_arrive_expect_tx(&full[stage], 2 * L::STAGE_BYTES);
          uint8_t* sa = smem + stage * L::STAGE_BYTES;
          tma_load_2d_pair(sa, ta, full_cl[stage], (int32_t)(kb * GBK), arow);
          if (bmn) {
#pragma unroll
            for (int j = 0; j < 2; ++j)  // box j: columns j*64.., k rows kb*64..
              tma_load_2d_pair(sa + L::A_BYTES + j * (64 * GBK * 2), tb, full_cl[stage],
                               bcol + j * 64, (int32_t)(kb * GBK));
          } else {
            tma_load_2d_pair(sa + L::A_BYTES, tb, full_cl[stage], (int32_t)(kb * GBK), bcol);
          }
          ++issued;
          if (++stage == GPS) { stage = 0; ph ^= 1; }
        }
        if (!ok) break;
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
          for (uint32_t i = top > (uint32_t)GPS ? top - GPS : 0u; i < top; ++i) {
            const int s = (int)(i % GPS);
            const uint32_t par = (i / GPS) & 1u;
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
      int stage = 0;
      uint32_t ph = 0, acc = 0;
      uint32_t aph[2] = {0, 0};
      GUnit nu = u0 < u1 ? a.units[u0] : GUnit{};
      for (int ui = u0; ui < u1 && !*abort_flag; ++ui) {
        const GUnit u = nu;
        if (ui + 1 < u1) nu = a.units[ui + 1];
        const int64_t kbt = u.kbf >> 1;
        const bool bmn = (u.kbf & 1) != 0;
        const uint32_t idesc =
            bmn ? tc::idesc_bf16_f32_bmn(256, 256) : tc::idesc_bf16_f32(256, 256);
        if (!tc::mbar_wait(&tempty[acc], aph[acc] ^ 1, w)) break;
        tc::tc_fence_after();
        const uint32_t d = tmem_base + acc * 256;
        bool ok = true;
        for (int64_t kb = 0; kb < kbt; ++kb) {
          if (!tc::mbar_wait(&full[stage], ph, w)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
          const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < GBK / 16; ++kk) {
            const uint64_t db = bmn ? tc::smem_desc_mn_sw128(sb + kk * 16 * 128, 64 * GBK * 2, 1024)
                                    : tc::smem_desc_sw128(sb + kk * 32);
            tc::mma_bf16_pair(d, tc::smem_desc_sw128(sa + kk * 32), db, idesc,
                              (kb > 0 || kk > 0) ? 1u : 0u);
          }
          tc::mma_commit_pair(&empty[stage]);
          if (++stage == GPS) { stage = 0; ph ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit_pair(&tfull[acc]);
        aph[acc] ^= 1;
        acc ^= 1;
      }
      tc::mma_commit_pair(drain);  // every MMA of the pair done (both CTAs' drain barriers)
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drain, 0) && clock64() - t0 < tc::kDrainCycles) {
      }
    }
  } else {
    const int q = warp & 3;
    uint32_t te[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) te[b] = tc::mapa_shared(&tempty[b], 0);
    grouped_epilogue<256, 256>(a, u0, u1, tmem_base, tfull, smem + L::EPI_OFF + q * 8192,
                               (int64_t)rank * 128, w, q, lane,
                               [&](uint32_t b) { tc::mbar_arrive_remote_relaxed(te[b]); });
  }
  __syncthreads();
  tc::tc_fence_before();
  tc::cluster_sync();  // no CTA leaves while its peer may still signal its barriers
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc_pair(tmem_base, 512);
}

template <int BMN, int BK, int TMN>
__global__ void __launch_bounds__(256) grouped_simt_kernel(GArgs a) {
  __shared__ __align__(16) SimtSmem<float, BMN, BMN, BK> sm;
  const int u0 = a.cta_off[blockIdx.x], u1 = a.cta_off[blockIdx.x + 1];
  for (int ui = u0; ui < u1; ++ui) {
    const GUnit u = a.units[ui];
    const GMeta& g = a.meta[u.p];
    simt_tile<float, BMN, BMN, BK, TMN, TMN>(
        static_cast<const float*>(g.A), g.lda, static_cast<const float*>(g.B), g.ldb,
        static_cast<float*>(g.C), g.ldc, g.m, g.n, (int64_t)u.tile_row * BMN,
        (int64_t)u.tile_col * BMN, 0, g.k, sm);
  }
}

// 128 x 128 tiles: the cp.async ring, 16-byte copies for problems whose rows
// allow them and 4-byte copies otherwise.
__global__ void __launch_bounds__(256) grouped_f32_kernel(GArgs a) {
  extern __shared__ __align__(16) uint8_t gsm[];
  const int u0 = a.cta_off[blockIdx.x], u1 = a.cta_off[blockIdx.x + 1];
  for (int ui = u0; ui < u1; ++ui) {
    const GUnit u = a.units[ui];
    const GMeta& g = a.meta[u.p];
    const float* A = static_cast<const float*>(g.A);
    const float* B = static_cast<const float*>(g.B);
    float* C = static_cast<float*>(g.C);
    const int64_t r0 = (int64_t)u.tile_row * 128, c0 = (int64_t)u.tile_col * 128;
    if (g.f32_async)
      f32_tile<128, 4>(A, g.lda, B, g.ldb, C, g.ldc, g.m, g.n, r0, c0, 0, g.k, g.vec_ok != 0,
                       *reinterpret_cast<F32Smem<128>*>(gsm));
    else
      f32_tile<128, 1>(A, g.lda, B, g.ldb, C, g.ldc, g.m, g.n, r0, c0, 0, g.k, g.vec_ok != 0,
                       *reinterpret_cast<F32Smem<128>*>(gsm));
  }
}

// ---- host -----------------------------------------------------------------------

int encode(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
           int box_rows) {
  return encode_tmap_bf16(map, base, rows, cols, ld, GBK, box_rows);
}

int pick_tile(int count, const cosma_problem* pr, int dtype, int requested) {
  if (dtype == COSMA_BF16) {
    if (requested == 128 || requested == 256 || requested == 512) return requested;
    std::vector<int64_t> ns(count);
    for (int i = 0; i < count; ++i) ns[i] = pr[i].n;
    std::nth_element(ns.begin(), ns.begin() + count / 2, ns.end());
    return ns[count / 2] >= 512 ? 256 : 128;
  }
  // f32: the 128 x 128 cp.async tile (about three times the FFMA rate of the
  // 64 x 64 one even on small problems); 64 only on request.
  if (requested == 64 || requested == 128) return requested;
  return 128;
}

bool needs_pack(const cosma_problem& q) {
  return (reinterpret_cast<uintptr_t>(q.A) & 15) || ((q.lda * 2) & 15);
}
bool b_direct(const cosma_problem& q) {
  return (reinterpret_cast<uintptr_t>(q.B) & 15) == 0 && ((q.ldb * 2) & 15) == 0;
}
bool c_tensor_store(const cosma_problem& q) {
  return (reinterpret_cast<uintptr_t>(q.C) & 15) == 0 && ((q.ldc * 4) & 15) == 0;
}

// f32 C map for tensor stores: 32 x 32 boxes, 128-byte swizzle.
int encode_c(CUtensorMap* map, void* base, int64_t rows, int64_t cols, int64_t ld) {
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
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COSMA_OK : COSMA_ERR_CUDA;
}

long long ws_need(int count, const cosma_problem* pr, int dtype) {
  if (dtype != COSMA_BF16) return 0;
  long long b = 0;
  for (int i = 0; i < count; ++i) {
    const cosma_problem& q = pr[i];
    if (!(q.m > 0 && q.n > 0 && q.k > 0)) continue;
    if (!b_direct(q)) b += rup(q.n * rup(q.k, 8) * 2, 256);
    if (needs_pack(q)) b += rup(q.m * rup(q.k, 8) * 2, 256);
  }
  return b;
}

// Builds (or finds) the device table of this group.
int get_table(int dev, int count, const cosma_problem* pr, int dtype, int tile, int sms, void* ws,
              bool capturing, cudaStream_t st, Table** out) {
  unsigned long long key = mix(0, (unsigned long long)count);
  key = mix(key, (unsigned long long)dtype);
  key = mix(key, (unsigned long long)tile);
  key = mix(key, (unsigned long long)(uintptr_t)ws);
  for (int i = 0; i < count; ++i) {
    const cosma_problem& q = pr[i];
    key = mix(key, (unsigned long long)q.m);
    key = mix(key, (unsigned long long)q.n);
    key = mix(key, (unsigned long long)q.k);
    key = mix(key, (unsigned long long)(uintptr_t)q.A);
    key = mix(key, (unsigned long long)q.lda);
    key = mix(key, (unsigned long long)(uintptr_t)q.B);
    key = mix(key, (unsigned long long)q.ldb);
    key = mix(key, (unsigned long long)(uintptr_t)q.C);
    key = mix(key, (unsigned long long)q.ldc);
  }
  for (int s = 0; s < kCacheSlots; ++s) {
    Table& t = g_cache[dev][s];
    if (t.dev && t.key == key && t.count == count && t.dtype == dtype && t.tile_n == tile) {
      if (capturing) t.captured = true;
      *out = &t;
      return COSMA_OK;
    }
  }
  if (capturing) return COSMA_ERR_NO_WORKSPACE;

  // Host image of the table.  tile 512 (bf16): 256 x 256 tiles on CTA pairs, each CTA
  // loading 128-row boxes of A and of a transposed B.
  const bool pair = dtype == COSMA_BF16 && tile == 512;
  const int tm = GBM;
  const int tn = pair ? 256 : tile;
  const int tmm = dtype == COSMA_BF16 ? (pair ? 256 : tm) : tile;
  std::vector<GMeta> meta(count);
  std::vector<GMap> maps(dtype == COSMA_BF16 ? count : 0);
  std::vector<int64_t> tpre(count + 1, 0);
  std::vector<int64_t> apre(count + 1, 0);
  std::vector<GUnit> units;
  std::vector<int64_t> cost;
  uint8_t* wsp = static_cast<uint8_t*>(ws);
  for (int i = 0; i < count; ++i) {
    const cosma_problem& q = pr[i];
    GMeta& g = meta[i];
    g.m = q.m; g.n = q.n; g.k = q.k;
    g.A = q.A; g.lda = q.lda; g.B = q.B; g.ldb = q.ldb; g.C = q.C; g.ldc = q.ldc;
    g.Bt = nullptr; g.ldt = 0; g.Ap = nullptr; g.ldap = 0;
    g.b_mn = 0; g.c_tma = 0;
    g.f32_async = ((reinterpret_cast<uintptr_t>(q.A) & 15) == 0 && (q.lda & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(q.B) & 15) == 0 && (q.ldb & 3) == 0)
                      ? 1
                      : 0;
    apre[i + 1] = apre[i];
    g.vec_ok = ((reinterpret_cast<uintptr_t>(q.C) & 15) == 0 && (q.ldc & 3) == 0) ? 1 : 0;
    if (dtype == COSMA_BF16 && q.m > 0 && q.n > 0 && q.k > 0) {
      const int64_t kp = rup(q.k, 8);
      g.b_mn = b_direct(q) ? 1 : 0;
      if (!g.b_mn) {
        g.Bt = reinterpret_cast<__nv_bfloat16*>(wsp);
        g.ldt = kp;
        wsp += rup(q.n * kp * 2, 256);
      }
      const void* a_src = q.A;
      int64_t a_ld = q.lda;
      if (needs_pack(q)) {
        g.Ap = reinterpret_cast<__nv_bfloat16*>(wsp);
        g.ldap = kp;
        wsp += rup(q.m * kp * 2, 256);
        a_src = g.Ap;
        a_ld = kp;
        apre[i + 1] = apre[i] + ((q.m + PT - 1) / PT) * ((q.k + PT - 1) / PT);
      }
      int rc = encode(&maps[i].ta, a_src, q.m, q.k, a_ld, GBM);
      if (rc != COSMA_OK) return rc;
      if (g.b_mn) {  // B itself: k rows of n, 64 x 64 boxes
        rc = encode_tmap_bf16(&maps[i].tb, q.B, q.k, q.n, q.ldb, 64, GBK);
        tpre[i + 1] = tpre[i];
      } else {
        rc = encode(&maps[i].tb, g.Bt, q.n, q.k, kp, pair ? 128 : tn);
        tpre[i + 1] = tpre[i] + ((q.n + PT - 1) / PT) * ((q.k + PT - 1) / PT);
      }
      if (rc != COSMA_OK) return rc;
      if (c_tensor_store(q) && q.n >= 4) {
        rc = encode_c(&maps[i].tc, q.C, q.m, q.n & ~(int64_t)3, q.ldc);
        if (rc != COSMA_OK) return rc;
        g.c_tma = 1;
      }
    }
    if (dtype == COSMA_BF16 && !(q.m > 0 && q.n > 0 && q.k > 0)) tpre[i + 1] = tpre[i];
    if (q.m == 0 || q.n == 0 || q.k == 0) continue;
    const int64_t mt = (q.m + tmm - 1) / tmm, nt = (q.n + tn - 1) / tn;
    for (int64_t r = 0; r < mt; ++r)
      for (int64_t c = 0; c < nt; ++c) {
        units.push_back(GUnit{i, (int)r, (int)c, (int)(((q.k + 63) / 64) << 1 | g.b_mn)});
        cost.push_back((q.k + 63) / 64 + 2);  // k blocks + epilogue
      }
  }
  // Longest-processing-time-first assignment of units to CTAs.
  const int64_t U = (int64_t)units.size();
  // (for pair tiles, "ctas" counts CTA pairs)
  const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(pair ? std::max(1, sms / 2) : sms, U));
  std::vector<int64_t> order(U);
  for (int64_t i = 0; i < U; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return cost[x] > cost[y]; });
  typedef std::pair<int64_t, int> Load;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int c = 0; c < ctas; ++c) heap.push(Load(0, c));
  std::vector<std::vector<int64_t>> per(ctas);
  for (int64_t oi = 0; oi < U; ++oi) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(order[oi]);
    l.first += cost[order[oi]];
    heap.push(l);
  }
  std::vector<GUnit> flat;
  flat.reserve(U);
  std::vector<int> off(ctas + 1, 0);
  for (int c = 0; c < ctas; ++c) {
    // Each CTA runs its units in reverse assignment order, cheapest first: the
    // CTAs' j-th units from the end are neighbours in the cost-sorted,
    // problem-major list -- mostly tiles of one problem -- so concurrent CTAs share
    // that problem's panels in L2.  Measured on one GB300 (512 log-uniform bf16
    // products): most expensive first 757 TFLOP/s, heavy and light alternating
    // 777, cheapest first 801.
    for (size_t i = per[c].size(); i-- > 0;) flat.push_back(units[per[c][i]]);
    off[c + 1] = (int)flat.size();
  }

  // Device image: [maps][meta][units][cta_off][tprefix]
  size_t o_maps = 0;
  size_t o_meta = rup((int64_t)(maps.size() * sizeof(GMap)), 256);
  size_t o_units = o_meta + rup((int64_t)(meta.size() * sizeof(GMeta)), 256);
  size_t o_off = o_units + rup((int64_t)(std::max<int64_t>(U, 1) * sizeof(GUnit)), 256);
  size_t o_tp = o_off + rup((int64_t)((ctas + 1) * sizeof(int)), 256);
  size_t o_ap = o_tp + rup((int64_t)((count + 1) * sizeof(int64_t)), 256);
  size_t total = o_ap + rup((int64_t)((count + 1) * sizeof(int64_t)), 256);
  std::vector<uint8_t> host(total, 0);
  if (!maps.empty()) memcpy(host.data() + o_maps, maps.data(), maps.size() * sizeof(GMap));
  memcpy(host.data() + o_meta, meta.data(), meta.size() * sizeof(GMeta));
  if (U) memcpy(host.data() + o_units, flat.data(), flat.size() * sizeof(GUnit));
  memcpy(host.data() + o_off, off.data(), off.size() * sizeof(int));
  memcpy(host.data() + o_tp, tpre.data(), tpre.size() * sizeof(int64_t));
  memcpy(host.data() + o_ap, apre.data(), apre.size() * sizeof(int64_t));

  Table& t = g_cache[dev][g_next[dev]];
  g_next[dev] = (g_next[dev] + 1) % kCacheSlots;
  if (t.captured) {  // a graph may still read it: keep it, take a fresh buffer
    g_retired[dev].push_back(t.dev);
    t = Table{};
  }
  if (t.dev && t.bytes < total) {
    cudaFree(t.dev);  // synchronising free of an older group's table
    t.dev = nullptr;
  }
  if (!t.dev) {
    if (cudaMalloc(&t.dev, total) != cudaSuccess) {
      cudaGetLastError();
      t = Table{};
      return COSMA_ERR_NO_WORKSPACE;
    }
    t.bytes = total;
  }
  // Ordered on the call's stream, after earlier launches that may still read
  // this slot's previous table (the pageable source is staged before return).
  if (cudaMemcpyAsync(t.dev, host.data(), total, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(t.dev);
    t = Table{};
    return COSMA_ERR_CUDA;
  }
  uint8_t* d = static_cast<uint8_t*>(t.dev);
  t.key = key;
  t.count = count;
  t.dtype = dtype;
  t.tile_n = tile;
  t.ctas = ctas;
  t.maps = reinterpret_cast<const GMap*>(d + o_maps);
  t.meta = reinterpret_cast<const GMeta*>(d + o_meta);
  t.units = reinterpret_cast<const GUnit*>(d + o_units);
  t.cta_off = reinterpret_cast<const int*>(d + o_off);
  t.tprefix = reinterpret_cast<const int64_t*>(d + o_tp);
  t.aprefix = reinterpret_cast<const int64_t*>(d + o_ap);
  t.ttiles = tpre[count];
  t.atiles = apre[count];
  t.nunits = U;
  *out = &t;
  return COSMA_OK;
}

template <int BN, int STAGES>
int launch_tc(const Table& t, const GArgs& args, cudaStream_t st) {
  using L = GLayout<BN, STAGES>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(grouped_tc_kernel<BN, STAGES>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC);
  });
  if (attr != cudaSuccess) return (int)attr;
  prof_mark(st, true);
  grouped_tc_kernel<BN, STAGES><<<t.ctas, 192, L::ALLOC, st>>>(args);
  prof_mark(st, false);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_pair(const Table& t, const GArgs& args, cudaStream_t st) {
  using L = GPairLayout;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(grouped_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                L::ALLOC);
  });
  if (attr != cudaSuccess) return (int)attr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * t.ctas));
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = L::ALLOC;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  prof_mark(st, true);
  const cudaError_t le = cudaLaunchKernelEx(&cfg, grouped_pair_kernel, args);
  prof_mark(st, false);
  if (le != cudaSuccess) return (int)le;
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace

int grouped_gemm(int count, const cosma_problem* problems, int dtype, const DeviceInfo& dev,
                 void* ws, long long ws_bytes, int* status, long long wait_limit,
                 cudaStream_t st, long long* needed, int requested_tile) {
  const long long need = ws_need(count, problems, dtype);
  if (needed) {  // sizing pass: report the workspace, launch nothing
    *needed = need;
    return COSMA_OK;
  }
  if (need > ws_bytes) return COSMA_ERR_NO_WORKSPACE;
  const int tile = pick_tile(count, problems, dtype, requested_tile);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
  // The launch reads a copy of the slot's host-side fields taken under the lock,
  // so another host thread rebuilding the slot cannot tear them mid-read.  The
  // device tables those fields point to are not protected by the copy: grouped
  // calls must not overlap across streams (include/cosma.h).
  Table snap;
  int rc;
  {
    std::lock_guard<std::mutex> lock(g_tab_mu);
    Table* slot = nullptr;
    rc = get_table(dev.device, count, problems, dtype, tile, dev.sms > 0 ? dev.sms : 148, ws,
                   cs != cudaStreamCaptureStatusNone, st, &slot);
    if (rc == COSMA_OK) snap = *slot;
  }
  if (rc != COSMA_OK) return rc;
  const Table* t = &snap;
  if (t->nunits == 0) return COSMA_OK;
  GArgs args{t->maps, t->meta, t->units, t->cta_off, status, wait_limit};
  if (dtype == COSMA_BF16) {
    if (t->ttiles + t->atiles > 0) {
      const int64_t blocks = std::min<int64_t>(t->ttiles + t->atiles,
                                               (int64_t)(dev.sms > 0 ? dev.sms : 148) * 16);
      grouped_prep_kernel<<<(unsigned)blocks, 256, 0, st>>>(
          t->meta, t->tprefix, t->aprefix, count, t->ttiles, t->atiles);
      count_launch();
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return (int)e;
    }
    if (tile == 512) return launch_pair(*t, args, st);
    return tile == 256 ? launch_tc<256, 4>(*t, args, st) : launch_tc<128, 6>(*t, args, st);
  }
  if (tile == 128) {
    static cudaError_t attr = cudaFuncSetAttribute(
        grouped_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(F32Smem<128>));
    if (attr != cudaSuccess) return (int)attr;
    prof_mark(st, true);
    grouped_f32_kernel<<<t->ctas, 256, sizeof(F32Smem<128>), st>>>(args);
  } else {
    prof_mark(st, true);
    grouped_simt_kernel<64, 16, 4><<<t->ctas, 256, 0, st>>>(args);
  }
  prof_mark(st, false);
  count_launch();
  return (int)cudaGetLastError();
}

void grouped_release(int dev) {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  if (dev < 0 || dev >= 16) return;
  for (int s = 0; s < kCacheSlots; ++s) {
    if (g_cache[dev][s].dev) cudaFree(g_cache[dev][s].dev);
    g_cache[dev][s] = Table{};
  }
  for (void* p : g_retired[dev]) cudaFree(p);
  g_retired[dev].clear();
  g_next[dev] = 0;
}

}  // namespace cosma

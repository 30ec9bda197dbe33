// Host planner: Alg. 1's FindSeqSchedule -> ParallelizeSched -> FitRanks
// mapped onto one GPU (processors = SMs, S = one SM's fast memory).
//
//   find_seq_schedule   the Sec. 5.2 problem max ab/(a+b) s.t. ab + a + 1 <= S,
//                       solved over integers (the printed eq. aopt/bopt is its
//                       continuous optimum floored and can be off by one).
//   fit_ranks_weighted  Sec. 7.1: processor grid [pm, pn, pk] with at most
//                       floor(delta p) idle processors minimising the words of
//                       one local domain; the weights scale the A, B and C
//                       faces (all 1 for the paper's element-granular form).
//   plan_gemm           picks, for the kernel family of a dtype, the C tile
//                       (largest intensity rho = ab/(a+b) among the tiles the
//                       kernel implements, shrunk when (mnk/P)^(1/3) is small --
//                       eq. optTileShape), the k split pk and the assignment
//                       order, by an explicit cost model (below).
//   sched_from_plan     the work-unit schedule of a plan, including the raster
//                       group of the tiles in flight (the square-tile rule one
//                       level up, with L2 as the fast memory of the wave).
#include <math.h>
#include <string.h>
#include <algorithm>

#include "internal.h"

namespace cosma {

namespace {

const double kClockHz = 1.9e9;        // sustained SM clock assumed by the cost model
const double kHbmBytesPerS = 6.5e12;  // device HBM bandwidth
const double kL2BytesPerClkSm = 64.0; // L2 -> SM bandwidth per SM
const double kLaunchS = 4e-6;         // one kernel launch + tail

struct TileChoice {
  int tile_m, tile_n, k_block, stages;
  double eff = 1.0;  // main-loop efficiency of this tile relative to its family's
};

// Tiles each kernel family implements.
int tiles_for(int kernel, TileChoice* out) {
  switch (kernel) {
    case COSMA_KERNEL_SIMT_F64:
      out[0] = {128, 128, 8, 2}; out[1] = {64, 64, 8, 2};
      return 2;
    case COSMA_KERNEL_SIMT_F32:
      // 256 x 128 runs 512 threads at a 128-register cap; 128 x 256 (16 columns
      // per thread) measured 7 % faster per tile than 128 x 128 at 16384^3 and
      // 65536^2 x 1024, and loses where its fewer tiles leave a partial last wave
      out[0] = {128, 128, 32, 4, 1.0}; out[1] = {256, 128, 32, 4, 0.95};
      out[2] = {128, 256, 32, 4, 1.07};
      return 3;
    case COSMA_KERNEL_TC_BF16:
      out[0] = {128, 256, 64, 4}; out[1] = {128, 128, 64, 6};
      return 2;
    case COSMA_KERNEL_EMU_BF16:
      // 256-row tiles run on CTA pairs (2 SMs per tile); MMAs 128 columns wide
      // reach about 81 % of the per-clock rate of 256-wide ones
      out[0] = {256, 256, 64, 7, 1.0}; out[1] = {128, 128, 64, 5, 0.81};
      out[2] = {256, 128, 64, 9, 0.81};
      return 3;
    case COSMA_KERNEL_TF32X3:  // k blocks of 32 f32 (one 128-byte row); C sums in registers
      out[0] = {128, 128, 32, 3};
      return 1;
  }
  return 0;
}

KernelDesc desc_for(int dtype, const DeviceInfo& dev) {
  KernelDesc d{};
  const double smem = dev.smem_per_sm > 0 ? dev.smem_per_sm : 233472.0;
  const double rf = dev.regs_per_sm > 0 ? dev.regs_per_sm * 4.0 : 262144.0;
  const double tmem = 262144.0;
  switch (dtype) {
    case COSMA_F64:
      d.kernel = COSMA_KERNEL_SIMT_F64; d.w_in = 8; d.w_acc = 8; d.w_out = 8;
      d.fast_bytes = smem + rf; d.flops_per_clk_sm = 4.0; d.efficiency = 0.9;
      break;
    case COSMA_F32:
      d.kernel = COSMA_KERNEL_SIMT_F32; d.w_in = 4; d.w_acc = 4; d.w_out = 4;
      d.fast_bytes = smem + rf; d.flops_per_clk_sm = 256.0; d.efficiency = 0.6;
      break;
    case COSMA_BF16:
      d.kernel = COSMA_KERNEL_TC_BF16; d.w_in = 2; d.w_acc = 4; d.w_out = 4;
      d.fast_bytes = smem + tmem; d.flops_per_clk_sm = 8192.0; d.efficiency = 0.8;
      break;
    case COSMA_F32_EMU_TF32:  // three tf32 products at half the bf16 rate
      d.kernel = COSMA_KERNEL_TF32X3; d.w_in = 4; d.w_acc = 4; d.w_out = 4;
      d.fast_bytes = smem + tmem; d.flops_per_clk_sm = 4096.0 / 3.0; d.efficiency = 0.8;
      break;
    default:  // emulated FP64: bf16 slices
      d.kernel = COSMA_KERNEL_EMU_BF16; d.w_in = 2; d.w_acc = 8; d.w_out = 8;
      d.fast_bytes = smem + tmem; d.flops_per_clk_sm = 8192.0; d.efficiency = 0.7;
      break;
  }
  return d;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

int find_seq_schedule(long long S, int* a_out, int* b_out) {
  if (S < 3 || !a_out || !b_out) return COSMA_ERR_INVALID_ARG;
  // For fixed a the intensity ab/(a+b) grows with b, so only b = floor((S-a-1)/a)
  // can be optimal; compare candidates exactly as rationals.
  long long best_a = 0, best_b = 0;
  for (long long a = 1; 2 * a + 1 <= S; ++a) {
    const long long b = (S - a - 1) / a;
    if (b < 1) break;
    if (best_a == 0) { best_a = a; best_b = b; continue; }
    const __int128 lhs = (__int128)(a * b) * (best_a + best_b);
    const __int128 rhs = (__int128)(best_a * best_b) * (a + b);
    if (lhs > rhs || (lhs == rhs && a * b < best_a * best_b)) { best_a = a; best_b = b; }
  }
  if (best_a == 0) return COSMA_ERR_INVALID_ARG;
  *a_out = (int)best_a;
  *b_out = (int)best_b;
  return COSMA_OK;
}

int fit_ranks_weighted(int64_t m, int64_t n, int64_t k, int p, double delta, double wa,
                       double wb, double wc, int grid[3]) {
  if (m < 1 || n < 1 || k < 1 || p < 1 || !(delta >= 0.0) || delta >= 1.0 || !grid)
    return COSMA_ERR_INVALID_ARG;
  const long long min_used = p - (long long)floor(delta * (double)p);
  long double best = -1.0L;
  int bm = 0, bn = 0, bk = 0;
  // Processors used, most first; inside, grids in lexicographic order.  Only a
  // strictly smaller word count replaces the incumbent, which gives the tie rule.
  for (long long used = p; used >= std::max(1LL, min_used); --used) {
    for (long long pm = 1; pm <= std::min<long long>(m, used); ++pm) {
      if (used % pm) continue;
      const long long rest = used / pm;
      for (long long pn = 1; pn <= std::min<long long>(n, rest); ++pn) {
        if (rest % pn) continue;
        const long long pk = rest / pn;
        if (pk > k) continue;
        const long double lm = (long double)cdiv(m, pm), ln = (long double)cdiv(n, pn),
                          lk = (long double)cdiv(k, pk);
        const long double words = wa * lm * lk + wb * lk * ln + wc * lm * ln;
        if (best < 0.0L || words < best) {
          best = words; bm = (int)pm; bn = (int)pn; bk = (int)pk;
        }
      }
    }
  }
  if (bm == 0) return COSMA_ERR_INVALID_ARG;
  grid[0] = bm; grid[1] = bn; grid[2] = bk;
  return COSMA_OK;
}

long long workspace_bytes(int64_t m, int64_t n, int64_t k, int dtype, const cosma_plan& p) {
  auto align = [](long long x) { return (x + 255) / 256 * 256; };
  long long bytes = 0;
  const int w_acc = (dtype == COSMA_F32 || dtype == COSMA_BF16 || dtype == COSMA_F32_EMU_TF32) ? 4 : 8;
  if (p.pk > 1) bytes += align((long long)p.pk * m * n * w_acc);
  if (dtype == COSMA_BF16) bytes += align((long long)n * k * 2);  // B^T (k-major) copy
  return bytes;
}

Sched sched_from_plan(int64_t m, int64_t n, int64_t k, const cosma_plan& p) {
  Sched s{};
  s.m = m; s.n = n; s.k = k;
  s.tile_m = p.tile_m; s.tile_n = p.tile_n; s.k_block = p.k_block;
  s.mt = cdiv(m, p.tile_m); s.nt = cdiv(n, p.tile_n); s.kbt = cdiv(k, p.k_block);
  s.pm = p.pm; s.pn = p.pn; s.pk = p.pk; s.order = p.order; s.ctas = p.ctas;
  // Raster group of order 1 (rows of tiles per group): the ctas / pk tiles in flight
  // at once form a G x W block.  One k step of that wave reads G tile_m rows of A and
  // W tile_n columns of B through L2; with G W fixed the sum is smallest at
  // G tile_m = W tile_n -- the square-tile rule of eq. optTileShape one level up,
  // L2 being the fast memory of the whole wave.  (The emulated FP64 kernels run
  // the units of one k slice together: their wave is ctas tiles.)
  {
    const bool emu = p.kernel == COSMA_KERNEL_EMU_BF16;
    const double wave = std::max(1.0, (double)p.ctas / (emu ? 1 : std::max(1, p.pk)));
    int g = (int)std::lround(std::sqrt(wave * p.tile_n / std::max(1, p.tile_m)));
    if (g < 1) g = 1;
    if (g > s.mt) g = (int)std::max<int64_t>(1, s.mt);
    s.group = g;
  }
  return s;
}

// Estimated seconds of one decomposition (see file header).
static double estimate(const KernelDesc& d, int64_t m, int64_t n, const TileChoice& t,
                       int64_t max_units, int64_t kblocks_per_unit, int pk) {
  const double flops_kb = 2.0 * t.tile_m * t.tile_n * t.k_block;
  const double t_compute = flops_kb / (d.flops_per_clk_sm * d.efficiency * t.eff * kClockHz);
  const double t_io = (double)(t.tile_m + t.tile_n) * t.k_block * d.w_in /
                      (kL2BytesPerClkSm * kClockHz);
  const double t_kb = std::max(t_compute, t_io);
  const double t_epi = (double)t.tile_m * t.tile_n * (pk > 1 ? d.w_acc : d.w_out) /
                       (kL2BytesPerClkSm * kClockHz);
  double s = (double)max_units * ((double)kblocks_per_unit * t_kb + t_epi) + kLaunchS;
  if (pk > 1) s += (2.0 * pk + 1.0) * m * n * d.w_acc / kHbmBytesPerS + kLaunchS;
  return s;
}

static void finish_plan(int64_t m, int64_t n, int64_t k, int dtype, const KernelDesc& d, int P,
                        cosma_plan& best) {
  const int64_t mm = std::max<int64_t>(m, 1), nn = std::max<int64_t>(n, 1);
  best.kernel = d.kernel;
  best.sms = P;
  best.fast_words = d.fast_bytes / d.w_in;
  // Listing-1 I/O of the schedule: each tile streams k (h + w) input words and
  // writes h w outputs; a k split adds pk partial stores + pk loads + 1 store.
  const int64_t mt = cdiv(mm, best.tile_m), ntl = cdiv(nn, best.tile_n);
  double io = (double)k * ((double)ntl * m + (double)mt * n);
  io += (double)m * n * (best.pk > 1 ? 2.0 * best.pk + 1.0 : 1.0);
  best.io_words = io;
  best.bound_words = 2.0 * (double)m * n * k / sqrt(best.fast_words) + (double)m * n;
  best.workspace_bytes = workspace_bytes(m, n, k, dtype, best);
}

int plan_candidate(int64_t m, int64_t n, int64_t k, int dtype, int c, const DeviceInfo& dev,
                   const cosma_config& cfg, cosma_plan* out) {
  if (!out || m < 1 || n < 1 || k < 1 || c < 0 || c >= COSMA_MLP_OUT) return COSMA_ERR_INVALID_ARG;
  if (dtype < COSMA_F64 || dtype > COSMA_F64_EMU_BF16) return COSMA_ERR_INVALID_ARG;
  const KernelDesc d = desc_for(dtype, dev);
  const int P = dev.sms > 0 ? dev.sms : 148;
  TileChoice tiles[4];
  const int ntiles = tiles_for(d.kernel, tiles);
  const int ti = (c / 8) % 2;
  if (ti >= ntiles) return COSMA_ERR_UNSUPPORTED;
  const int pks[4] = {1, 2, 4, 8};
  const int pk = pks[(c / 2) % 4];
  const int order = c % 2;
  const TileChoice& t = tiles[ti];
  const int64_t mt = cdiv(m, t.tile_m), ntl = cdiv(n, t.tile_n), kbt = cdiv(k, t.k_block);
  if (pk > kbt) return COSMA_ERR_UNSUPPORTED;
  if (d.kernel == COSMA_KERNEL_EMU_BF16 && (pk != 1 || order != 1)) return COSMA_ERR_UNSUPPORTED;
  cosma_plan p{};
  p.tile_m = t.tile_m; p.tile_n = t.tile_n; p.k_block = t.k_block; p.stages = t.stages;
  p.pk = pk; p.order = order;
  const int64_t kbu = cdiv(kbt, pk);
  int64_t mu;
  const bool pair = d.kernel == COSMA_KERNEL_EMU_BF16 && t.tile_m == 256;
  if (order == 1) {
    const int64_t units = mt * ntl * pk;
    p.pm = p.pn = 1;
    p.ctas = (int)std::min<int64_t>(pair ? std::max(1, P / 2) : P, units);
    mu = cdiv(units, p.ctas);
  } else {
    int g[3];
    if (fit_ranks_weighted(mt, ntl, 1, std::max(1, P / pk), cfg.delta,
                           (double)t.tile_m * t.k_block * kbu * d.w_in,
                           (double)t.k_block * kbu * t.tile_n * d.w_in,
                           (double)t.tile_m * t.tile_n * d.w_acc, g) != COSMA_OK)
      return COSMA_ERR_UNSUPPORTED;
    p.pm = g[0]; p.pn = g[1];
    p.ctas = g[0] * g[1] * pk;
    mu = cdiv(mt, g[0]) * cdiv(ntl, g[1]);
  }
  TileChoice per_sm = t;
  if (pair) per_sm.tile_m = 128;
  p.est_seconds = estimate(d, m, n, per_sm, mu, kbu, pk) * (pair ? 0.8 : 1.0);
  finish_plan(m, n, k, dtype, d, P, p);
  *out = p;
  return COSMA_OK;
}

int plan_gemm(int64_t m, int64_t n, int64_t k, int dtype, int selector, const DeviceInfo& dev,
              const cosma_config& cfg, cosma_plan* out, bool may_sync) {
  if (!out || m < 0 || n < 0 || k < 0) return COSMA_ERR_INVALID_ARG;
  if (dtype < COSMA_F64 || dtype > COSMA_F32_EMU_TF32) return COSMA_ERR_INVALID_ARG;
  if (dtype == COSMA_F64_EMU_INT8) return COSMA_ERR_UNSUPPORTED;
  if (selector == COSMA_SELECT_LEARNED) {
    const int rc = learned_plan(m, n, k, dtype, dev, cfg, out, may_sync);
    if (rc == COSMA_OK) return rc;  // otherwise fall back to the analytic plan
  }
  const KernelDesc d = desc_for(dtype, dev);
  const int P = dev.sms > 0 ? dev.sms : 148;
  const int64_t mm = std::max<int64_t>(m, 1), nn = std::max<int64_t>(n, 1),
                kk = std::max<int64_t>(k, 1);
  TileChoice tiles[4];
  const int nt_choices = tiles_for(d.kernel, tiles);

  // ParallelizeSched (eq. optTileShape): the local domain side (mnk/P)^(1/3).
  // Tiles much larger than it would leave SMs idle; they stay candidates and
  // the cost model below decides.
  double best_s = -1.0;
  cosma_plan best{};
  for (int ti = 0; ti < nt_choices; ++ti) {
    const TileChoice& t = tiles[ti];
    const int64_t mt = cdiv(mm, t.tile_m), ntl = cdiv(nn, t.tile_n), kbt = cdiv(kk, t.k_block);
    const int64_t tiles_total = mt * ntl;
    // Candidate k splits: 1, powers of two while the units stay within 16 waves
    // (a split also evens out the last, partial wave of tiles), and the one that
    // fills the SMs when tiles are few.
    // The emulated FP64 kernels split k at super-chunk boundaries (4096 k), into
    // 2 .. 16 slices: enough to even out the last wave of pair tiles.
    int pks[16];
    int npk = 0;
    pks[npk++] = 1;
    const bool emu = d.kernel == COSMA_KERNEL_EMU_BF16;
    const int64_t nch = cdiv(kbt, kEmuChunkKb);
    if (!emu) {
      for (int pk = 2; pk <= 64 && npk < 16; pk *= 2)
        if (pk <= kbt && tiles_total * pk <= 16LL * P) pks[npk++] = pk;
      const int64_t fill = cdiv(P, tiles_total);
      if (fill > 1 && fill <= kbt && npk < 16) pks[npk++] = (int)fill;
    } else {
      for (int pk = 2; pk <= 16 && npk < 16; ++pk)
        if (pk <= nch) pks[npk++] = pk;
    }
    for (int pi = 0; pi < npk; ++pi) {
      const int pk = pks[pi];
      const int64_t kbu = emu ? std::min<int64_t>(kbt, cdiv(nch, pk) * kEmuChunkKb) : cdiv(kbt, pk);
      // order 1: balanced stripes (a 256-row emulation tile occupies a pair of SMs)
      {
        const bool pair = d.kernel == COSMA_KERNEL_EMU_BF16 && t.tile_m == 256;
        const int64_t units = tiles_total * pk;
        const int ctas = (int)std::min<int64_t>(pair ? std::max(1, P / 2) : P, units);
        const int64_t mu = cdiv(units, ctas);
        TileChoice per_sm = t;
        if (pair) per_sm.tile_m = 128;
        const double s = estimate(d, m, n, per_sm, mu, kbu, pk) * (pair ? 0.8 : 1.0);
        if (best_s < 0 || s < best_s) {
          best_s = s;
          best = cosma_plan{};
          best.tile_m = t.tile_m; best.tile_n = t.tile_n; best.k_block = t.k_block;
          best.stages = t.stages; best.pm = 1; best.pn = 1; best.pk = pk; best.order = 1;
          best.ctas = ctas;
        }
      }
      // order 0: the paper's grid, FitRanks over tiles x k slices
      if (d.kernel != COSMA_KERNEL_EMU_BF16) {
        const int p_plane = std::max(1, P / pk);
        int g[3];
        if (fit_ranks_weighted(mt, ntl, 1, p_plane, cfg.delta,
                               (double)t.tile_m * t.k_block * kbu * d.w_in,
                               (double)t.k_block * kbu * t.tile_n * d.w_in,
                               (double)t.tile_m * t.tile_n * d.w_acc, g) == COSMA_OK) {
          const int64_t mu = cdiv(mt, g[0]) * cdiv(ntl, g[1]);
          const double s = estimate(d, m, n, t, mu, kbu, pk);
          if (s < best_s) {
            best_s = s;
            best = cosma_plan{};
            best.tile_m = t.tile_m; best.tile_n = t.tile_n; best.k_block = t.k_block;
            best.stages = t.stages; best.pm = g[0]; best.pn = g[1]; best.pk = pk; best.order = 0;
            best.ctas = g[0] * g[1] * pk;
          }
        }
      }
    }
  }
  best.est_seconds = best_s;
  finish_plan(m, n, k, dtype, d, P, best);
  *out = best;
  return COSMA_OK;
}

int validate_plan(int64_t m, int64_t n, int64_t k, int dtype, const DeviceInfo& dev,
                  const cosma_plan& p) {
  const KernelDesc d = desc_for(dtype, dev);
  if (p.kernel != d.kernel) return COSMA_ERR_INVALID_ARG;
  TileChoice tiles[4];
  const int nt = tiles_for(d.kernel, tiles);
  bool ok = false;
  for (int i = 0; i < nt; ++i)
    if (tiles[i].tile_m == p.tile_m && tiles[i].tile_n == p.tile_n &&
        tiles[i].k_block == p.k_block)
      ok = true;
  if (!ok) return COSMA_ERR_INVALID_ARG;
  if (p.pk < 1 || p.ctas < 1 || p.order < 0 || p.order > 1) return COSMA_ERR_INVALID_ARG;
  const int64_t kbt = cdiv(std::max<int64_t>(k, 1), p.k_block);
  if (p.pk > kbt) return COSMA_ERR_INVALID_ARG;
  // emulated FP64: order 1, each k slice at least one super-chunk
  if (d.kernel == COSMA_KERNEL_EMU_BF16 &&
      (p.order != 1 || p.pk > cdiv(kbt, kEmuChunkKb)))
    return COSMA_ERR_INVALID_ARG;
  if (p.order == 0) {
    if (p.pm < 1 || p.pn < 1 || (long long)p.pm * p.pn * p.pk != p.ctas) return COSMA_ERR_INVALID_ARG;
    if (p.pm > cdiv(std::max<int64_t>(m, 1), p.tile_m) || p.pn > cdiv(std::max<int64_t>(n, 1), p.tile_n))
      return COSMA_ERR_INVALID_ARG;
  }
  if (p.ctas > 65535 * 4) return COSMA_ERR_INVALID_ARG;
  return COSMA_OK;
}

}  // namespace cosma

extern "C" int cosma_find_seq_schedule(long long S, int* a, int* b) {
  return cosma::find_seq_schedule(S, a, b);
}

extern "C" int cosma_fit_ranks(int64_t m, int64_t n, int64_t k, int p, double delta, int grid[3]) {
  return cosma::fit_ranks_weighted(m, n, k, p, delta, 1.0, 1.0, 1.0, grid);
}

// Work-unit decoding shared by the host planner (cosma_plan_units) and the
// kernels.  A work unit is one C tile over one k slice: the paper's local
// domain (Sec. 6.1) is the set of units one CTA (= one processor) executes.
//
// Two assignment orders:
//   order 0 -- rectangular local domains of the processor grid [pm, pn, pk]
//              (Alg. 1 GetDataDecomp): CTA c owns tile rows, tile columns and a
//              k slice, balanced to within one tile / one k block.
//   order 1 -- balanced stripes: units are enumerated in a blocked raster
//              (groups of `group` tile rows, columns inside a group) with the
//              pk k slices of a tile adjacent, and CTA c executes units
//              c, c + ctas, c + 2 ctas, ...  Concurrent CTAs then work on
//              neighbouring tiles, which share A rows and B columns in L2.
// The emulated FP64 kernels use order 1 with the k split outermost instead
// (emu_unit_of_cta): the units of one k range run together, and each range is
// a whole number of super-chunks.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define COSMA_HD __host__ __device__ __forceinline__
#else
#define COSMA_HD inline
#endif

namespace cosma {

struct Sched {
  int64_t m, n, k;     // problem
  int tile_m, tile_n;  // C tile
  int k_block;         // k granularity of slices
  int64_t mt, nt, kbt; // tiles along m, n; k blocks along k
  int pm, pn, pk;      // processor grid (order 0) / k split (both orders)
  int order;
  int ctas;
  int group;           // raster group height in tiles (order 1)
};

struct Unit {
  int64_t tile_row, tile_col;  // tile coordinates
  int64_t kb0, kb1;            // k-block range [kb0, kb1)
  int ks;                      // k slice index in [0, pk)
};

COSMA_HD int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Balanced split of `total` items into `parts`: start of part i.
COSMA_HD int64_t split_start(int64_t total, int64_t parts, int64_t i) {
  return (total / parts) * i + (i < total % parts ? i : total % parts);
}

// Number of units CTA `cta` executes.
COSMA_HD int64_t units_of_cta(const Sched& s, int cta) {
  if (s.order == 0) {
    const int im = cta / (s.pn * s.pk), in = (cta / s.pk) % s.pn;
    const int64_t rows = split_start(s.mt, s.pm, im + 1) - split_start(s.mt, s.pm, im);
    const int64_t cols = split_start(s.nt, s.pn, in + 1) - split_start(s.nt, s.pn, in);
    return rows * cols;
  }
  const int64_t total = s.mt * s.nt * s.pk;
  return cta < total ? (total - cta + s.ctas - 1) / s.ctas : 0;
}

// Tile number `tile` of the order-1 raster: groups of `group` tile rows, the
// columns of a group one after another, rows inside a column.
COSMA_HD void raster_tile(const Sched& s, int64_t tile, Unit& u) {
  const int64_t g = tile / ((int64_t)s.group * s.nt);
  const int64_t rows_in_group =
      (s.mt - g * s.group) < s.group ? (s.mt - g * s.group) : (int64_t)s.group;
  const int64_t idx = tile - g * (int64_t)s.group * s.nt;
  u.tile_col = idx / rows_in_group;
  u.tile_row = g * s.group + idx % rows_in_group;
}

// The i-th unit of CTA `cta` (0 <= i < units_of_cta).
COSMA_HD Unit unit_of_cta(const Sched& s, int cta, int64_t i) {
  Unit u;
  if (s.order == 0) {
    const int im = cta / (s.pn * s.pk), in = (cta / s.pk) % s.pn, ik = cta % s.pk;
    const int64_t r0 = split_start(s.mt, s.pm, im), r1 = split_start(s.mt, s.pm, im + 1);
    const int64_t c0 = split_start(s.nt, s.pn, in);
    const int64_t rows = r1 - r0;
    u.tile_row = r0 + i % rows;   // column of tiles at a time: the B panel stays hot
    u.tile_col = c0 + i / rows;
    u.ks = ik;
  } else {
    const int64_t unit = cta + i * (int64_t)s.ctas;
    u.ks = (int)(unit % s.pk);
    raster_tile(s, unit / s.pk, u);
  }
  u.kb0 = split_start(s.kbt, s.pk, u.ks);
  u.kb1 = split_start(s.kbt, s.pk, u.ks + 1);
  return u;
}

// The k-block range of the i-th unit of CTA `cta` alone -- what the MMA issuer
// needs -- without decoding the tile (whose 64-bit divisions would otherwise
// sit between two units' MMAs).
COSMA_HD void unit_k_range(const Sched& s, int cta, int64_t i, int64_t& kb0, int64_t& kb1) {
  if (s.pk == 1) {
    kb0 = 0;
    kb1 = s.kbt;
    return;
  }
  const int ks = s.order == 0 ? cta % s.pk : (int)((cta + i * (int64_t)s.ctas) % s.pk);
  kb0 = split_start(s.kbt, s.pk, ks);
  kb1 = split_start(s.kbt, s.pk, ks + 1);
}

// Super-chunk of the emulated FP64 kernels, in 64-wide k blocks (4096 k): the
// k extent over which their int32 level sums stay exact for every slice
// configuration they accept (at most 8 slices of at most 8 bits).
constexpr int kEmuChunkKb = 64;

// k-block range of k slice ks of an emulated FP64 plan: the super-chunks are
// split evenly over the pk slices, so every slice sums whole super-chunks --
// the ones an unsplit product would sum -- and the split changes no bit of C.
COSMA_HD void emu_k_range(const Sched& s, int ks, int64_t& kb0, int64_t& kb1) {
  const int64_t nch = cdiv64(s.kbt, kEmuChunkKb);
  kb0 = split_start(nch, s.pk, ks) * kEmuChunkKb;
  kb1 = split_start(nch, s.pk, ks + 1) * kEmuChunkKb;
  if (kb1 > s.kbt) kb1 = s.kbt;
}

// The i-th unit of CTA `cta` of an emulated FP64 plan (order 1): units are
// numbered k slice first, so concurrent CTAs share one k range and read the
// same slice panels from L2.
COSMA_HD Unit emu_unit_of_cta(const Sched& s, int cta, int64_t i) {
  Unit u;
  const int64_t unit = cta + i * (int64_t)s.ctas;
  const int64_t tiles = s.mt * s.nt;
  u.ks = (int)(unit / tiles);
  raster_tile(s, unit - (int64_t)u.ks * tiles, u);
  emu_k_range(s, u.ks, u.kb0, u.kb1);
  return u;
}

}  // namespace cosma

// Geometry of the tile-upper layout shared by its stream (tc_sym.cu) and the
// ||A_off||_F^2 pass of the objective: 128 x 128 tiles of the nd x nd matrix,
// tile (I, J) stored for J >= I only, in the order the stream visits them.
#pragma once

#include "common.cuh"

namespace nsrgs {

constexpr int kTsTile = 128;
constexpr int kTsTileBytes = kTsTile * kTsTile * 2;  // bfloat16 tile: 32 KB
constexpr int kTs8TileBytes = kTsTile * kTsTile;     // FP8-E4M3 tile: 16 KB

__host__ __device__ inline int ts_tile_rows(int n, int d) { return (int)(((long long)n * d + kTsTile - 1) / kTsTile); }
__host__ __device__ inline long long ts_tiles(int NT) { return (long long)NT * (NT + 1) / 2; }

// Tile width (MMA N) of the tensor-core stream for block size d <= 64: X^T tiles
// carry N rows, the ones past d zero.
__host__ __device__ constexpr int ts_width(int d) { return d <= 16 ? 16 : (d <= 32 ? 32 : 64); }

// Row tiles per strip (and per group) of the processing order (by tile width): as many as the
// stream's TMEM holds, R row accumulators plus two column buffers of 512
// columns (FP8 at d <= 32 keeps its hi and lo products side by side: 2d each).
__host__ __device__ constexpr int ts_strip_rows(int d, bool f8) { return d == 64 ? 4 : (f8 && d == 32 ? 6 : 8); }

// Byte offset of element (r, c) inside a 128-byte-swizzled bfloat16 128 x 128
// tile, and of element (n, k) (n < N rows, k < 128) inside an N x 128 X^T tile:
// 8-row groups 2048 bytes apart, the two 64-column halves 1024 bytes apart, rows
// 128 bytes apart, 16-byte chunk k of a row at k ^ (r % 8).
__host__ __device__ inline int ts_swz(int r, int c) {
  const int s = c >> 6, k = (c & 63) >> 3, e = c & 7;
  return (r >> 3) * 2048 + s * 1024 + (r & 7) * 128 + ((k ^ (r & 7)) << 4) + e * 2;
}

// The same for one-byte elements: a row is one 128-byte swizzle row, 8-row
// groups 1024 bytes apart, 16-byte chunk k (16 elements) of row r at k ^ (r % 8).
__host__ __device__ inline int ts8_swz(int r, int c) {
  return (r >> 3) * 1024 + (r & 7) * 128 + (((c >> 4) ^ (r & 7)) << 4) + (c & 15);
}

// Row r (0..127) of the element at byte offset o of a one-byte swizzled tile.
__host__ __device__ inline int ts8_row_of(int o) { return (o >> 10) * 8 + ((o >> 7) & 7); }

// Processing order: groups of R row tiles (I0 = g R), inside a group the
// columns J = I0 .. NT-1, inside a column ("strip") the rows I = I0 .. min(I0 +
// R, J + 1, NT) - 1.  Each tile appears once.
template <int R>
struct TsWalk {
  int NT, g, I0, Rg, J, r;
  __device__ int strip_len() const { return min(Rg, J - I0 + 1); }
  __device__ void set_group(int gg) {
    g = gg;
    I0 = g * R;
    Rg = min(R, NT - I0);
    J = I0;
    r = 0;
  }
  // Position of tile number t of the processing order.
  __device__ void seek(long long t) {
    long long base = 0;
    int gg = 0;
    for (;; ++gg) {
      const int L = NT - gg * R, Rgg = min(R, L);
      const long long cnt = (long long)Rgg * (Rgg + 1) / 2 + (long long)(L - Rgg) * Rgg;
      if (t < base + cnt) break;
      base += cnt;
    }
    set_group(gg);
    long long u = t - base;
    const long long tri = (long long)Rg * (Rg + 1) / 2;  // strips of 1, 2, .., Rg tiles, then Rg each
    if (u < tri) {
      int c = 0;
      while (u >= c + 1) {
        u -= c + 1;
        ++c;
      }
      J = I0 + c;
      r = (int)u;
    } else {
      u -= tri;
      J = I0 + Rg + (int)(u / Rg);
      r = (int)(u % Rg);
    }
  }
  __device__ int I() const { return I0 + r; }
  // Advances; reports whether the tile just left closed its strip / its group.
  __device__ void next(bool& strip_end, bool& group_end) {
    strip_end = group_end = false;
    if (++r < strip_len()) return;
    strip_end = true;
    r = 0;
    if (++J < NT) return;
    group_end = true;
    set_group(g + 1);
  }
};

// Byte offset of the FP8 per-block-row scales (float[n]) behind the tiles.
__host__ __device__ inline long long ts8_scale_offset(int n, int d) {
  return ts_tiles(ts_tile_rows(n, d)) * (long long)kTs8TileBytes;
}

}  // namespace nsrgs

// Y = A_off X on the tensor cores reading only the upper triangle of A, for
// 8 < d <= 64 with A stored in bfloat16 (NSRGS_BF16 at these d) or in FP8-E4M3
// with one float32 scale per block row (NSRGS_FP8E4M3 at these d).  The MMA's N
// is the tile width ts_width(d) (16, 32 or 64); X^T rows past d are zero, and
// where d does not divide 128 blocks straddle tiles (a stored tile keeps the
// elements with block(row) < block(col), so nothing needs a special case).
//
// Layout ("tile-upper"): the nd x nd matrix is cut into 128 x 128 tiles; tile
// (I, J) is stored for J >= I only, in the order the kernel visits them (groups
// of R row tiles, columns J inside a group, rows inside a column; see TsWalk),
// so that every CTA streams one contiguous range of the buffer.
// A diagonal tile keeps the blocks strictly above the block diagonal (d divides
// 128, so blocks never straddle tiles); everything else in it is zero.  Each
// tile is already in the 128-byte-swizzled order the tensor core reads (32 KB
// in bfloat16, 16 KB in E4M3: ts_swz / ts8_swz).  FP8 storage keeps
// q_ij = RN(A_ij / s_i) with s_i = max_{j > i} max |A_ij| / 448 (the rule of the
// FP8 panels), the n scales behind the tiles.
// One tile feeds both products of the symmetric form:
//   Y_I += A_IJ X_J     (A_IJ as a K-major operand, M = 128 rows, K = 128 columns)
//   Y_J += A_IJ^T X_I   (the same bytes as an MN-major operand: M = 128 columns,
//                        K = 128 rows)
// X^T is stored per 128-row tile in the same swizzled order (N rows), so every
// copy is a plain 1-D bulk copy.  In bfloat16 it is X rounded to nearest.  With
// FP8 tiles both MMA operands are E4M3, so X travels as two E4M3 planes, hi =
// RN(g X) and lo = RN(g X - hi) with g a power of two that puts max |X| in
// [128, 256): hi + lo carries X to about 2^-8 relative, and both planes
// accumulate into the same TMEM columns.  The row product uses X (scale g_r;
// its result is multiplied by s_i / g_r per output row), the column product
// uses the rows s_i X_i (scale g_c, result times 1 / g_c): the block-row scale
// runs along K there, so it is folded into the operand instead of the result.
//
// Per CTA (7 warps, persistent over a contiguous range of the processing order):
// tiles are visited in column strips of R row tiles (a group of R row panels,
// columns J = I0 .. NT-1, rows I0 .. I0+R-1 in each column), so the column
// product accumulates over a whole strip (K = up to 128 R rows) before it is
// added to Y, and the row products of the R panels stay in TMEM over the group.
//   warp 0 lane 0 : producer.  cp.async.bulk of each tile into a ring of stages
//                   (as many as shared memory holds), of X_J^T into one of two
//                   slots when a strip starts (every tile of a strip shares J),
//                   and of the group's R X_I^T tiles into one buffer when a group
//                   starts; mbarrier expect_tx.
//   warp 1        : allocates TMEM (D1: R slots of N columns, D2: two buffers of
//                   N columns); lane 0 issues the row product's tcgen05.mma
//                   (D1[r] += A X_J over the tile's columns), commits the stage
//                   and, at a group's end, D1.
//   warp 6 lane 0 : issues the column product's tcgen05.mma (D2 += A^T X_I over
//                   the tile's rows), commits the stage and, at a strip's end, D2.
//                   A stage is free once both issuers committed it.  With one
//                   thread issuing both products a tile took about 2000 cycles of
//                   that thread (the issue itself, not the tensor pipe, bound the
//                   stream); descriptors are base + constant offsets.
//   warps 2..5    : epilogue.  tcgen05.ld of their 32-lane quarter of D2 (rows =
//                   the strip's columns) and of the used D1 slots, then
//                   red.global.add.v4.f32 into Y.
// Every wait is bounded; a timeout sets FLAG_TIMEOUT and the CTA still frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "src.cuh"
#include "tc_common.cuh"
#include "tc_sym.cuh"

namespace nsrgs {

// Threads per CTA: producer, row-product MMA issue, 4 epilogue warps, column-product MMA issue.
constexpr int kTsThreads = 224;

template <int N, bool F8>
struct TsCfg {
  static constexpr int TILE = F8 ? kTs8TileBytes : kTsTileBytes;
  static constexpr int R = ts_strip_rows(N, F8);         // row tiles per strip
  // FP8 at N <= 32: one MMA multiplies both X planes (B = the 2N rows hi, lo), the
  // two halves of the accumulator summed in the epilogue; at N = 64 the planes
  // take one MMA each into the same columns (TMEM holds no 2N-wide slots there).
  static constexpr bool MERGE = F8 && N <= 32;
  static constexpr int NACC = MERGE ? 2 * N : N;         // accumulator columns per slot
  static constexpr int XB = N * 256;                      // one X^T tile (FP8: hi and lo planes)
  static constexpr int STAGE = TILE;                      // the ring holds A tiles only
  static constexpr int SMEM_MAX = 227 * 1024;
  // as many stages as fit beside the two X_J^T slots and the group's R X_I^T tiles
  // Y staging of the epilogue: per warp its 32 rows as boxes of 32 rows x BW
  // floats (128 or 64 bytes per row, swizzled like the tensor map reads them)
  static constexpr int BW = N < 32 ? N : 32;
  static constexpr int BOX = 32 * BW * 4;
  static constexpr int STG_WARP = N * 128;
  static constexpr int STG = 4 * STG_WARP;
  static constexpr int NSTAGE_FIT = (SMEM_MAX - 1024 - 512 - (2 + R) * XB - STG) / STAGE;
  static constexpr int NSTAGE = NSTAGE_FIT > 12 ? 12 : NSTAGE_FIT;
  static constexpr int OFF_XJ = NSTAGE * STAGE;          // X_J^T of the current / next strip
  static constexpr int OFF_XI = OFF_XJ + 2 * XB;         // X^T of the group's R row tiles
  static constexpr int OFF_STG = OFF_XI + R * XB;       // Y staging, 4 warps
  static constexpr int OFF_BARS = OFF_STG + STG;
  static constexpr int NBARS = 2 * NSTAGE + 2 + 4 + 2 + 4;
  static constexpr int SMEM = 1024 + OFF_BARS + NBARS * 8 + 16;
  static constexpr int TMEM_NEED = (R + 2) * NACC;       // D1: R slots, D2: two buffers
  static constexpr int TMEM_COLS = TMEM_NEED <= 64 ? 64 : (TMEM_NEED <= 128 ? 128 : (TMEM_NEED <= 256 ? 256 : 512));
  // D1 += A X_J and D2 += A^T X_I (A read MN-major)
  static constexpr uint32_t IDESC_ROW = F8 ? tc8_idesc(128, NACC, false) : tc_idesc(128, N, false);
  static constexpr uint32_t IDESC_COL = F8 ? tc8_idesc(128, NACC, true) : tc_idesc(128, N, true);
  static_assert(STAGE % 1024 == 0 && XB % 1024 == 0 && (N * 128) % 1024 == 0 && STG_WARP % 1024 == 0,
                "1024-byte swizzle alignment");
  static_assert(NSTAGE >= 3, "pipeline depth");
  static_assert(SMEM <= SMEM_MAX, "shared memory");
  static_assert(TMEM_NEED <= 512, "tensor memory");
};

struct TsArgs {
  const uint8_t* tiles;  // packed tiles
  const uint8_t* xt;     // swizzled X^T tiles for the row product (NT x N*256 bytes)
  const uint8_t* xc;     // for the column product (the same as xt in bfloat16; rows s_i X_i in FP8)
  const float* rscale;   // FP8: per-block-row scales s_i
  float* Y;              // padded, zero on entry
  const int* skip;
  Ctl* ctl;
  int rows;              // n * d
  int NT;
  int D;                 // block size d <= N (Y and X rows hold d floats; X^T rows past d are zero)
};

// FP8 operand scale: g = 2^(7 - floor(log2 m)) puts m = max |value| in [128, 256)
// (m = 0: g = 1); `inverse` returns 1 / g.  Exponents are clamped so that g and
// 1 / g stay normal floats.
__device__ __forceinline__ float ts8_pow2(unsigned mbits, bool inverse) {
  if (mbits == 0u) return 1.f;
  int e = (int)((mbits >> 23) & 0xffu) - 127;
  e = max(-100, min(e, 120));
  return __uint_as_float((uint32_t)(inverse ? 127 - 7 + e : 127 + 7 - e) << 23);
}

// Shared-memory descriptor of (base + off): the start address sits in the low
// 14 bits as address / 16 and every operand lies below 256 KB, so offsets add
// to a base descriptor without a carry.
__device__ __forceinline__ uint64_t desc_at(uint64_t base, uint32_t off) { return base + (uint64_t)(off >> 4); }

template <int N, bool F8>
__global__ void __launch_bounds__(kTsThreads, 1) tc_sym_kernel(const __grid_constant__ CUtensorMap tmY, const TsArgs a) {
  using C = TsCfg<N, F8>;
  constexpr int R = C::R;
  if (*a.skip) return;  // uniform: written only by earlier launches
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::OFF_BARS);
  uint64_t* empty = full + C::NSTAGE;
  uint64_t* xi_full = empty + C::NSTAGE;
  uint64_t* xi_empty = xi_full + 1;
  uint64_t* d2_full = xi_empty + 1;   // [2]
  uint64_t* d2_empty = d2_full + 2;   // [2]
  uint64_t* d1_full = d2_empty + 2;
  uint64_t* d1_empty = d1_full + 1;
  uint64_t* xj_full = d1_empty + 1;   // [2]
  uint64_t* xj_empty = xj_full + 2;   // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xj_empty + 2);
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = ts_tiles(a.NT);
  const long long t0 = total * blockIdx.x / gridDim.x;
  const long long t1 = total * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 2);  // released by both MMA issuers
    }
    mbar_init(xi_full, 1);
    mbar_init(xi_empty, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&d2_full[s], 1);
      mbar_init(&d2_empty[s], 4);
      mbar_init(&xj_full[s], 1);
      mbar_init(&xj_empty[s], 1);
    }
    mbar_init(d1_full, 1);
    mbar_init(d1_empty, 4);
    failed = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc_warp(tmem_slot, (uint32_t)C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tm_d1 = tmem;                         // + r * NACC
  const uint32_t tm_d2 = tmem + (uint32_t)(R * C::NACC);  // + db * NACC

  auto fail = [&]() {
    atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
    failed = 1;
  };

  // Descriptor bases: A K-major (row product), A MN-major (column product), X^T
  // operands (K-major).  Rows of 128 bytes; 8-row groups 1024 (FP8) or 2048
  // (bfloat16, two 64-column halves 1024 apart) bytes apart.
  constexpr uint32_t GRP = F8 ? 1024 : 2048;
  const uint32_t s0 = smem_u32(smem);

  if (t0 < t1 && warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int st = 0, p = 0;
    uint32_t ph = 0;
    const uint64_t pol = l2_evict_first_policy();
    long long it = 0, kx = 0;  // tiles issued, strips started
    bool group_start = true, strip_start = true;
    for (long long t = t0; t < t1 && !failed; ++t, ++it) {
      if (group_start) {  // X^T of the group's row tiles (one buffer: wait for the previous group)
        if (p >= 1 && !mbar_wait_bounded(xi_empty, (uint32_t)((p - 1) & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(xi_full, (uint32_t)(w.Rg * C::XB));
        bulk_g2s(smem + C::OFF_XI, a.xc + (long long)w.I0 * C::XB, (uint32_t)(w.Rg * C::XB), xi_full);
        ++p;
      }
      if (strip_start) {  // X_J^T once per strip, two slots (wait for the strip two back)
        const int xs = (int)(kx & 1);
        if (kx >= 2 && !mbar_wait_bounded(&xj_empty[xs], (uint32_t)(((kx - 2) >> 1) & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(&xj_full[xs], C::XB);
        bulk_g2s(smem + C::OFF_XJ + xs * C::XB, a.xt + (long long)w.J * C::XB, C::XB, &xj_full[xs]);
        ++kx;
      }
      if (it >= C::NSTAGE && !mbar_wait_bounded(&empty[st], ph ^ 1u, kWaitLimitNs)) {
        fail();
        break;
      }
      mbar_arrive_expect_tx(&full[st], C::STAGE);
      bulk_g2s_hint(smem + st * C::STAGE, a.tiles + t * (long long)C::TILE, C::TILE, &full[st], pol);
      if (++st == C::NSTAGE) {
        st = 0;
        ph ^= 1u;
      }
      bool se, ge;
      w.next(se, ge);
      group_start = ge;
      strip_start = se;
    }
    // Do not leave while copies into this CTA's shared memory may be in flight.
    const long long first = it > C::NSTAGE ? it - C::NSTAGE : 0;
    for (long long k = first; k < it; ++k)
      if (!mbar_wait_bounded(&full[k % C::NSTAGE], (uint32_t)((k / C::NSTAGE) & 1), kWaitLimitNs)) break;
    for (long long k = kx > 2 ? kx - 2 : 0; k < kx; ++k)
      mbar_wait_bounded(&xj_full[k & 1], (uint32_t)((k >> 1) & 1), kWaitLimitNs);
    if (p >= 1) mbar_wait_bounded(xi_full, (uint32_t)((p - 1) & 1), kWaitLimitNs);
  } else if (t0 < t1 && warp == 1 && lane == 0) {
    // ------------------------------------------------ row-product MMA issue
    // D1[r] += A_IJ X_J for the tile's row r of the group; X_J^T per strip.
    const uint64_t dA = sw128_desc(s0, 16, GRP), dX = sw128_desc(s0 + C::OFF_XJ, 16, GRP);
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int st = 0, p = 0;
    uint32_t ph = 0;
    long long k = 0;  // strips started
    bool group_start = true, strip_start = true;
    uint32_t started = 0;  // D1 slots written in this group segment
    for (long long t = t0; t < t1 && !failed; ++t) {
      if (group_start) {
        if (p >= 1 && !mbar_wait_bounded(d1_empty, (uint32_t)((p - 1) & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        started = 0;
      }
      const int xs = (int)(k & 1);
      if (strip_start && !mbar_wait_bounded(&xj_full[xs], (uint32_t)((k >> 1) & 1), kWaitLimitNs)) {
        fail();
        break;
      }
      if (!mbar_wait_bounded(&full[st], ph, kWaitLimitNs)) {
        fail();
        break;
      }
      tc_fence_after();
      const int r = w.r;
      const uint32_t d = tm_d1 + (uint32_t)(r * C::NACC);
      const uint64_t a0 = desc_at(dA, (uint32_t)(st * C::STAGE)), x0 = desc_at(dX, (uint32_t)(xs * C::XB));
      const uint32_t acc0 = (started >> r & 1u);
      if constexpr (C::MERGE) {
        // K = the tile's 128 columns: four K = 32 steps, B = X_J's hi and lo planes (2N rows)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc_mma8(d, desc_at(a0, kk * 32), desc_at(x0, kk * 32), C::IDESC_ROW, kk == 0 ? acc0 : 1u);
      } else if constexpr (F8) {
        // K = the tile's 128 columns: four K = 32 steps, hi and lo planes of X_J
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int pl = 0; pl < 2; ++pl)
            tc_mma8(d, desc_at(a0, kk * 32), desc_at(x0, pl * N * 128 + kk * 32), C::IDESC_ROW,
                    (kk == 0 && pl == 0) ? acc0 : 1u);
      } else {
        // K = the tile's 128 columns: two 64-column halves of four K = 16 steps
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            tc_mma(d, desc_at(a0, h * 1024 + kk * 32), desc_at(x0, h * 1024 + kk * 32), C::IDESC_ROW,
                   (h == 0 && kk == 0) ? acc0 : 1u);
      }
      started |= 1u << r;
      tc_commit(&empty[st]);
      if (++st == C::NSTAGE) {
        st = 0;
        ph ^= 1u;
      }
      bool se, ge;
      w.next(se, ge);
      const bool last = (t + 1 == t1);
      if (se || last) {
        tc_commit(&xj_empty[xs]);
        ++k;
      }
      if (ge || last) {
        tc_commit(d1_full);
        ++p;
      }
      strip_start = se;
      group_start = ge;
    }
  } else if (t0 < t1 && warp == kTsThreads / 32 - 1 && lane == 0) {
    // --------------------------------------------- column-product MMA issue
    // D2 += A_IJ^T X_I over the strip's rows (the same tile read MN-major).
    const uint64_t dA = sw128_desc(s0, 1024, GRP), dX = sw128_desc(s0 + C::OFF_XI, 16, GRP);
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int st = 0, p = 0;
    uint32_t ph = 0;
    long long k = 0;  // strips started
    bool group_start = true, strip_start = true;
    for (long long t = t0; t < t1 && !failed; ++t) {
      if (group_start && !mbar_wait_bounded(xi_full, (uint32_t)(p & 1), kWaitLimitNs)) {
        fail();
        break;
      }
      const int db = (int)(k & 1);
      if (strip_start && k >= 2 && !mbar_wait_bounded(&d2_empty[db], (uint32_t)(((k - 2) >> 1) & 1), kWaitLimitNs)) {
        fail();
        break;
      }
      if (!mbar_wait_bounded(&full[st], ph, kWaitLimitNs)) {
        fail();
        break;
      }
      tc_fence_after();
      const uint32_t d = tm_d2 + (uint32_t)(db * C::NACC);
      const uint64_t a0 = desc_at(dA, (uint32_t)(st * C::STAGE)), x0 = desc_at(dX, (uint32_t)(w.r * C::XB));
      const uint32_t acc0 = strip_start ? 0u : 1u;
      if constexpr (C::MERGE) {
        // K = the tile's 128 rows: four K = 32 steps of four 8-row groups, B = hi and lo planes
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc_mma8(d, desc_at(a0, kk * 4096), desc_at(x0, kk * 32), C::IDESC_COL, kk == 0 ? acc0 : 1u);
      } else if constexpr (F8) {
        // K = the tile's 128 rows: four K = 32 steps of four 8-row groups, hi and lo planes
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int pl = 0; pl < 2; ++pl)
            tc_mma8(d, desc_at(a0, kk * 4096), desc_at(x0, pl * N * 128 + kk * 32), C::IDESC_COL,
                    (kk == 0 && pl == 0) ? acc0 : 1u);
      } else {
        // K = the tile's 128 rows: eight K = 16 steps of two 8-row groups
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          tc_mma(d, desc_at(a0, kk * 4096), desc_at(x0, (kk >> 2) * 1024 + (kk & 3) * 32), C::IDESC_COL,
                 kk == 0 ? acc0 : 1u);
      }
      tc_commit(&empty[st]);
      if (++st == C::NSTAGE) {
        st = 0;
        ph ^= 1u;
      }
      bool se, ge;
      w.next(se, ge);
      const bool last = (t + 1 == t1);
      if (se || last) {
        tc_commit(&d2_full[db]);
        ++k;
      }
      if (ge || last) {
        tc_commit(xi_empty);
        ++p;
      }
      strip_start = se;
      group_start = ge;
    }
  } else if (t0 < t1 && warp >= 2 && warp < 6) {
    // -------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int p = 0;
    long long k = 0;
    uint32_t used = 0;  // D1 slots written in this group segment
    // FP8: the row product is scaled by s_i / g_r per output row, the column product by 1 / g_c
    float inv_gr = 1.f, inv_gc = 1.f;
    if constexpr (F8) {
      inv_gr = ts8_pow2(a.ctl->ts8_max[0], true);
      inv_gc = ts8_pow2(a.ctl->ts8_max[1], true);
    }
    // The warp's 32 rows go to Y through shared memory: swizzled 16-byte stores
    // (conflict-free: the 8 rows of a phase hit 8 different bank groups), then one
    // TMA reduce-add per 32 x BW box, rows past n*d clipped by the tensor map.
    // One red.global per row and 16 bytes cost about 2000 cycles per 32 KB drain.
    uint8_t* stg = smem + C::OFF_STG + (warp - 2) * C::STG_WARP;
    const uint32_t stg_s = smem_u32(stg);
    auto drain = [&](uint32_t taddr, int row, bool row_product) -> bool {  // TMEM rows 32q.. -> Y rows row..
      float v[C::NACC];
#pragma unroll
      for (int c0 = 0; c0 < C::NACC; c0 += 16) {
        float tt[16];
        tc_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, tt);
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c0 + c] = tt[c];
      }
      tc_wait_ld();
      if constexpr (C::MERGE) {
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] += v[N + c];  // A X_hi + A X_lo
      }
      if constexpr (F8) {
        const float m = row_product ? (row < a.rows ? a.rscale[row / a.D] : 0.f) * inv_gr : inv_gc;
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] *= m;
      }
      if (a.D != N) {  // d < N: rows of d floats, not 16-byte multiples; element-wise adds
        if (row < a.rows) {
          float* y = a.Y + (long long)row * a.D;
#pragma unroll
          for (int c = 0; c < N; ++c)
            if (c < a.D) red_add_f32(y + c, v[c]);
        }
        return true;
      }
      if (lane == 0) bulk_wait_read_all();  // the previous drain's boxes have left the staging
      __syncwarp();
      const int sw = C::BW == 32 ? (lane & 7) : ((lane >> 1) & 3);
#pragma unroll
      for (int c = 0; c < N / 4; ++c) {
        const int b = c / (C::BW / 4), k = c % (C::BW / 4);
        st_shared_v4(stg + b * C::BOX + lane * (C::BW * 4) + ((k ^ sw) << 4), v[4 * c], v[4 * c + 1], v[4 * c + 2],
                     v[4 * c + 3]);
      }
      fence_proxy_async_shared();
      __syncwarp();
      const int row0 = row - lane;
      if (lane == 0 && row0 < a.rows) {
#pragma unroll
        for (int b = 0; b < N / C::BW; ++b) tma_reduce_add_2d(&tmY, stg_s + b * C::BOX, b * C::BW, row0);
        bulk_commit_group();
      }
      return true;
    };
    for (long long t = t0; t < t1; ++t) {
      used |= 1u << w.r;
      const int J = w.J, I0 = w.I0;
      bool se, ge;
      w.next(se, ge);
      const bool last = (t + 1 == t1);
      if (se || last) {  // the strip's column partials: Y rows of column tile J
        const int db = (int)(k & 1);
        if (!mbar_wait_bounded(&d2_full[db], (uint32_t)((k >> 1) & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        tc_fence_after();
        drain(tm_d2 + (uint32_t)(db * C::NACC), J * kTsTile + 32 * q + lane, false);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&d2_empty[db]);
        ++k;
      }
      if (ge || last) {  // the group's row partials: Y rows of each used row tile
        if (!mbar_wait_bounded(d1_full, (uint32_t)(p & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        tc_fence_after();
        for (int r = 0; r < R; ++r)
          if (used >> r & 1u) drain(tm_d1 + (uint32_t)(r * C::NACC), (I0 + r) * kTsTile + 32 * q + lane, true);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(d1_empty);
        used = 0;
        ++p;
      }
    }
    if (lane == 0) bulk_wait_all();  // the reduce-adds into Y are complete
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_warp(tmem, (uint32_t)C::TMEM_COLS);
  }
}

// ------------------------------------------------------------ packing
// One CTA per tile (grid-stride): tile number t of the processing order, in
// 16-byte chunks (8 bfloat16 or 16 E4M3 consecutive columns of a row).
// FP8: element (R, C) is stored as RN(A_RC / s_{R / d}), saturated to +-448.
template <int R, bool F8, class Src>
__global__ void __launch_bounds__(256) ts_pack_kernel(Src src, int NT, int rows, int d, const float* scale,
                                                     uint8_t* out) {
  __shared__ int ij[2];
  const long long total = ts_tiles(NT);
  constexpr int TILE = F8 ? kTs8TileBytes : kTsTileBytes;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {
      TsWalk<R> w;
      w.NT = NT;
      w.seek(t);
      ij[0] = w.I();
      ij[1] = w.J;
    }
    __syncthreads();
    const int I = ij[0], J = ij[1];
    uint8_t* tile = out + t * (long long)TILE;
    for (int ch = threadIdx.x; ch < TILE / 16; ch += blockDim.x) {
      uint32_t w[4];
      int off;
      if constexpr (F8) {
        const int r = ch >> 3, c = (ch & 7) * 16;
        const long long Rr = (long long)I * kTsTile + r, Cc = (long long)J * kTsTile + c;
        const float s = Rr < rows ? scale[Rr / d] : 1.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t v = 0;
#pragma unroll
          for (int e = 0; e < 4; ++e)
            v |= (uint32_t)__nv_cvt_float_to_fp8(src(Rr, Cc + 4 * k + e) / s, __NV_SATFINITE, __NV_E4M3) << (8 * e);
          w[k] = v;
        }
        off = ts8_swz(r, c);
      } else {
        const int r = ch >> 4, c = (ch & 15) * 8;
        const long long Rr = (long long)I * kTsTile + r, Cc = (long long)J * kTsTile + c;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const __nv_bfloat16 lo = __float2bfloat16_rn(src(Rr, Cc + 2 * k));
          const __nv_bfloat16 hi = __float2bfloat16_rn(src(Rr, Cc + 2 * k + 1));
          w[k] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        off = ts_swz(r, c);
      }
      *reinterpret_cast<uint4*>(tile + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// X^T tiles: element (nn, k) of tile J is X[128 J + k][nn] in bfloat16 (zero past n*d
// rows and for nn >= D, the block size, up to the tile width N).
__global__ void __launch_bounds__(256) ts_xt_kernel(const float* __restrict__ X, uint8_t* __restrict__ xt, int rows,
                                                   int D, int N, int NT, const int* skip) {
  if (*skip) return;
  const long long chunks = (long long)NT * N * (kTsTile / 8);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < chunks;
       e += (long long)gridDim.x * blockDim.x) {
    const int J = (int)(e / (N * (kTsTile / 8)));
    const int rem = (int)(e % (N * (kTsTile / 8)));
    const int nn = rem / (kTsTile / 8), k0 = (rem % (kTsTile / 8)) * 8;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long r0 = (long long)J * kTsTile + k0 + 2 * k;
      const float a = (nn < D && r0 < rows) ? X[r0 * D + nn] : 0.f;
      const float b = (nn < D && r0 + 1 < rows) ? X[(r0 + 1) * D + nn] : 0.f;
      w[k] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
             ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
    }
    *reinterpret_cast<uint4*>(xt + (long long)J * N * 256 + ts_swz(nn, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// FP8 operands, pass 1: mx[0] = max |X|, mx[1] = max |s_i X_i| (float bits; zero on entry).
__global__ void __launch_bounds__(256) ts8_xmax_kernel(const float* __restrict__ X, const float* __restrict__ scale,
                                                      int rows, int D, unsigned* mx, const int* skip) {
  if (*skip) return;
  float m0 = 0.f, m1 = 0.f;
  const long long count = (long long)rows * D;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float x = X[e];
    m0 = fmaxf(m0, fabsf(x));
    m1 = fmaxf(m1, fabsf(x * scale[e / D / D]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&mx[0], __float_as_uint(m0));
    atomicMax(&mx[1], __float_as_uint(m1));
  }
}

__device__ __forceinline__ void ts8_split(float v, uint32_t& hi, uint32_t& lo, int sh) {
  const __nv_fp8_storage_t h = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  const __half_raw hr = __nv_cvt_fp8_to_halfraw(h, __NV_E4M3);
  const float r = v - __half2float(__half(hr));  // exact: hi is v to 4 significant bits
  hi |= (uint32_t)h << sh;
  lo |= (uint32_t)__nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3) << sh;
}

// FP8 operands, pass 2: per 128-row tile J, the row operand (g_r X) and the
// column operand (g_c s_i X_i) as hi and lo E4M3 planes of N x 128 bytes each
// (element (nn, k) = row 128 J + k, column nn; zero past n*d rows and for nn >= D).
__global__ void __launch_bounds__(256) ts8_xt_kernel(const float* __restrict__ X, const float* __restrict__ scale,
                                                    uint8_t* __restrict__ xt, uint8_t* __restrict__ xc, int rows,
                                                    int D, int N, int NT, const unsigned* mx, const int* skip) {
  if (*skip) return;
  const float gr = ts8_pow2(mx[0], false), gc = ts8_pow2(mx[1], false);
  const long long chunks = (long long)NT * 8 * N;  // (tile, 16-row chunk, column), column fastest
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < chunks;
       e += (long long)gridDim.x * blockDim.x) {
    const int nn = (int)(e % N);
    const long long tk = e / N;
    const int J = (int)(tk >> 3), k0 = (int)(tk & 7) * 16;
    uint32_t rh[4] = {0, 0, 0, 0}, rl[4] = {0, 0, 0, 0}, ch[4] = {0, 0, 0, 0}, cl[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const long long row = (long long)J * kTsTile + k0 + k;
      float x = 0.f, sx = 0.f;
      if (row < rows && nn < D) {
        x = X[row * D + nn];
        sx = x * scale[row / D];
      }
      ts8_split(x * gr, rh[k >> 2], rl[k >> 2], 8 * (k & 3));
      ts8_split(sx * gc, ch[k >> 2], cl[k >> 2], 8 * (k & 3));
    }
    const long long base = (long long)J * N * 256;
    const int o = ts8_swz(nn, k0);
    *reinterpret_cast<uint4*>(xt + base + o) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<uint4*>(xt + base + N * 128 + o) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<uint4*>(xc + base + o) = make_uint4(ch[0], ch[1], ch[2], ch[3]);
    *reinterpret_cast<uint4*>(xc + base + N * 128 + o) = make_uint4(cl[0], cl[1], cl[2], cl[3]);
  }
}

// ---------------------------------------------------------------- host
// Block sizes the tile-upper layout takes: any d <= 64 (tile width ts_width(d); BF16
// and FP8 storage use it above d = 8).
bool tc_sym_supported(int d) { return d >= 1 && d <= 64; }

long long tc_sym_bytes(int n, int d) { return ts_tiles(ts_tile_rows(n, d)) * (long long)kTsTileBytes; }

// FP8 tiles plus the n block-row scales.
long long tc_sym8_scale_offset(int n, int d) { return ts8_scale_offset(n, d); }
long long tc_sym8_bytes(int n, int d) { return ts8_scale_offset(n, d) + ((long long)n * 4 + 15) / 16 * 16; }

// Bytes of the swizzled X^T tiles for (n, d): bfloat16 one set, FP8 two (row and column operands).
long long tc_sym_xt_bytes(int n, int d) { return (long long)ts_tile_rows(n, d) * ts_width(d) * 256; }
long long tc_sym8_xt_bytes(int n, int d) { return 2 * tc_sym_xt_bytes(n, d); }

static PFN_cuTensorMapEncodeTiled_v12000 ts_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Y (rows x N float32, row-major) as the epilogue's reduce-add target: boxes of
// 32 rows x BW floats, swizzled as the staging is written.
template <int N, bool F8>
static cudaError_t y_map(CUtensorMap* tm, float* Y, int rows) {
  using C = TsCfg<N, F8>;
  auto fn = ts_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)N * 4};
  cuuint32_t box[2] = {(cuuint32_t)C::BW, 32};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Y, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        C::BW == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int N, bool F8>
static cudaError_t launch_ts(const TsArgs& a, cudaStream_t st, bool prepare) {
  using C = TsCfg<N, F8>;
  if (prepare) return cudaFuncSetAttribute(tc_sym_kernel<N, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  CUtensorMap tm{};  // Y as a TMA target when its rows are the tile width (d = N); unused otherwise
  if (a.D == N) {
    const cudaError_t e = y_map<N, F8>(&tm, a.Y, a.rows);
    if (e != cudaSuccess) return e;
  }
  const long long total = ts_tiles(a.NT);
  const int grid = (int)std::min<long long>(total, num_sms());
  tc_sym_kernel<N, F8><<<grid, kTsThreads, C::SMEM, st>>>(tm, a);
  return cudaGetLastError();
}

static cudaError_t launch_ts_any(int d, bool f8, const TsArgs& a, cudaStream_t st, bool prepare) {
  switch (ts_width(d)) {
    case 16: return f8 ? launch_ts<16, true>(a, st, prepare) : launch_ts<16, false>(a, st, prepare);
    case 32: return f8 ? launch_ts<32, true>(a, st, prepare) : launch_ts<32, false>(a, st, prepare);
    case 64: return f8 ? launch_ts<64, true>(a, st, prepare) : launch_ts<64, false>(a, st, prepare);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc_sym_prepare(int d, bool f8) {
  TsArgs a{};
  return launch_ts_any(d, f8, a, 0, true);
}

// BF16 tiles packed with block size d against X of `width` columns (the Stiefel
// form's p >= d); the visiting order's strip length must be the same for the
// two tile widths (tc_sym_width_ok), since it is part of the packed layout.
bool tc_sym_width_ok(int d, int width) {
  return width >= d && width <= 64 && ts_strip_rows(ts_width(width), false) == ts_strip_rows(ts_width(d), false);
}
long long tc_sym_xt_bytes_w(int n, int d, int width) { return (long long)ts_tile_rows(n, d) * ts_width(width) * 256; }

cudaError_t tc_sym_product_w(const void* packed, int n, int d, int width, const float* X, uint8_t* xt, float* Y,
                             Ctl* ctl, const int* skip, cudaStream_t st) {
  if (!tc_sym_width_ok(d, width)) return cudaErrorInvalidValue;
  const int NT = ts_tile_rows(n, d), N = ts_width(width);
  const long long chunks = (long long)NT * N * (kTsTile / 8);
  const int g = (int)std::min<long long>((chunks + 255) / 256, 4LL * num_sms());
  ts_xt_kernel<<<g, 256, 0, st>>>(X, xt, n * d, width, N, NT, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TsArgs a{reinterpret_cast<const uint8_t*>(packed), xt, xt, nullptr, Y, skip, ctl, n * d, NT, width};
  return launch_ts_any(width, false, a, st, false);
}

cudaError_t tc_sym_product(const void* packed, int n, int d, bool f8, const float* X, uint8_t* xt, float* Y,
                           Ctl* ctl, const int* skip, cudaStream_t st) {
  const int NT = ts_tile_rows(n, d), N = ts_width(d);
  const uint8_t* tiles = reinterpret_cast<const uint8_t*>(packed);
  if (!f8) {
    const long long chunks = (long long)NT * N * (kTsTile / 8);
    const int g = (int)std::min<long long>((chunks + 255) / 256, 4LL * num_sms());
    ts_xt_kernel<<<g, 256, 0, st>>>(X, xt, n * d, d, N, NT, skip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TsArgs a{tiles, xt, xt, nullptr, Y, skip, ctl, n * d, NT, d};
    return launch_ts_any(d, false, a, st, false);
  }
  const float* scale = reinterpret_cast<const float*>(tiles + ts8_scale_offset(n, d));
  uint8_t* xc = xt + tc_sym_xt_bytes(n, d);
  cudaError_t e = cudaMemsetAsync(ctl->ts8_max, 0, sizeof(ctl->ts8_max), st);
  if (e != cudaSuccess) return e;
  const long long count = (long long)n * d * d;
  ts8_xmax_kernel<<<(int)std::min<long long>((count + 255) / 256, 2LL * num_sms()), 256, 0, st>>>(
      X, scale, n * d, d, ctl->ts8_max, skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long chunks = (long long)NT * 8 * N;
  ts8_xt_kernel<<<(int)std::min<long long>((chunks + 255) / 256, 4LL * num_sms()), 256, 0, st>>>(
      X, scale, xt, xc, n * d, d, N, NT, ctl->ts8_max, skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  TsArgs a{tiles, xt, xc, scale, Y, skip, ctl, n * d, NT, d};
  return launch_ts_any(d, true, a, st, false);
}

// FP8: the caller has written the block-row scales at ts8_scale_offset(n, d).
template <class Src>
cudaError_t tc_sym_pack(Src src, int n, int d, bool f8, void* packed, cudaStream_t st) {
  const int NT = ts_tile_rows(n, d);
  const int g = (int)std::min<long long>(ts_tiles(NT), 8LL * num_sms());
  uint8_t* out = reinterpret_cast<uint8_t*>(packed);
  const float* scale = reinterpret_cast<const float*>(out + ts8_scale_offset(n, d));
  const int rows = n * d;
#define NSRGS_TS_PACK(DD)                                                                        \
  if (f8)                                                                                        \
    ts_pack_kernel<ts_strip_rows(DD, true), true><<<g, 256, 0, st>>>(src, NT, rows, d, scale, out);   \
  else                                                                                           \
    ts_pack_kernel<ts_strip_rows(DD, false), false><<<g, 256, 0, st>>>(src, NT, rows, d, scale, out);
  switch (ts_width(d)) {  // the visiting order follows the tile width
    case 16: NSRGS_TS_PACK(16) break;
    case 32: NSRGS_TS_PACK(32) break;
    case 64: NSRGS_TS_PACK(64) break;
    default: return cudaErrorInvalidValue;
  }
#undef NSRGS_TS_PACK
  return cudaGetLastError();
}
template cudaError_t tc_sym_pack<UpperSrc>(UpperSrc, int, int, bool, void*, cudaStream_t);
template cudaError_t tc_sym_pack<DenseSrc>(DenseSrc, int, int, bool, void*, cudaStream_t);
template cudaError_t tc_sym_pack<SeAugSrc>(SeAugSrc, int, int, bool, void*, cudaStream_t);

}  // namespace nsrgs

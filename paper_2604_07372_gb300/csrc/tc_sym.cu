// Y = A_off X on the tensor cores reading only the upper triangle of A, for
// d in {16, 32, 64} with A stored in bfloat16 (NSRGS_BF16 at these d).
//
// Layout ("tile-upper"): the nd x nd matrix is cut into 128 x 128 tiles; tile
// (I, J) is stored for J >= I only, in the order the kernel visits them (groups
// of R row tiles, columns J inside a group, rows inside a column; see TsWalk),
// so that every CTA streams one contiguous range of the buffer.
// A diagonal tile keeps the blocks strictly above the block diagonal (d divides
// 128, so blocks never straddle tiles); everything else in it is zero.  Each
// tile is 32 KB, already in the 128-byte-swizzled order the tensor core reads:
// 8-row groups 2048 bytes apart, inside a group the two 64-column halves 1024
// bytes apart, rows 128 bytes apart, 16-byte chunk k of row r at k ^ (r % 8).
// One tile feeds both products of the symmetric form:
//   Y_I += A_IJ X_J     (A_IJ as a K-major operand, M = 128 rows, K = 128 columns)
//   Y_J += A_IJ^T X_I   (the same bytes as an MN-major operand: M = 128 columns,
//                        K = 128 rows; MN atoms 1024 bytes apart, K groups 2048)
// X^T is rounded to bfloat16 and stored per 128-row tile in the same swizzled
// order (N rows of 256 bytes), so every copy is a plain 1-D bulk copy.
//
// Per CTA (6 warps, persistent over a contiguous range of the processing order):
// tiles are visited in column strips of R row tiles (a group of R row panels,
// columns J = I0 .. NT-1, rows I0 .. I0+R-1 in each column), so the column
// product accumulates over a whole strip (K = up to 128 R rows) before it is
// added to Y, and the row products of the R panels stay in TMEM over the group.
//   warp 0 lane 0 : producer.  cp.async.bulk of each tile (32 KB) with its X_J^T
//                   tile into a ring of stages, and of the group's R X_I^T tiles
//                   into one buffer when a group starts; mbarrier expect_tx.
//   warp 1        : allocates TMEM (D1: R slots of N columns, D2: two buffers of
//                   N columns); lane 0 issues tcgen05.mma (eight K = 16 steps for
//                   D1[r] += A X_J, eight for D2 += A^T X_I) and commits the
//                   stage, D2 at a strip's end and D1 at a group's end.
//   warps 2..5    : epilogue.  tcgen05.ld of their 32-lane quarter of D2 (rows =
//                   the strip's columns) and of the used D1 slots, then
//                   red.global.add.v4.f32 into Y.
// Every wait is bounded; a timeout sets FLAG_TIMEOUT and the CTA still frees TMEM.
#include <algorithm>

#include "src.cuh"
#include "tc_common.cuh"

namespace nsrgs {

constexpr int kTsTile = 128;
constexpr int kTsTileBytes = kTsTile * kTsTile * 2;  // 32 KB

__host__ __device__ inline int ts_tile_rows(int n, int d) { return (int)(((long long)n * d + kTsTile - 1) / kTsTile); }
__host__ __device__ inline long long ts_tiles(int NT) { return (long long)NT * (NT + 1) / 2; }

// Byte offset of element (r, c) inside a swizzled 128 x 128 tile, and of
// element (n, k) (n < N rows, k < 128) inside a swizzled N x 128 X^T tile.
__host__ __device__ inline int ts_swz(int r, int c) {
  const int s = c >> 6, k = (c & 63) >> 3, e = c & 7;
  return (r >> 3) * 2048 + s * 1024 + (r & 7) * 128 + ((k ^ (r & 7)) << 4) + e * 2;
}

template <int N>
struct TsCfg {
  static constexpr int R = N == 64 ? 4 : 8;              // row tiles per strip
  static constexpr int XB = N * 256;                      // one X^T tile
  static constexpr int STAGE = kTsTileBytes + XB;        // A tile + X_J^T tile
  static constexpr int NSTAGE = N == 16 ? 5 : 3;
  static constexpr int OFF_XI = NSTAGE * STAGE;          // X^T of the group's R row tiles
  static constexpr int OFF_BARS = OFF_XI + R * XB;
  static constexpr int NBARS = 2 * NSTAGE + 2 + 4 + 2;
  static constexpr int SMEM = 1024 + OFF_BARS + NBARS * 8 + 16;
  static constexpr int TMEM_NEED = (R + 2) * N;          // D1: R slots, D2: two buffers
  static constexpr int TMEM_COLS = TMEM_NEED <= 64 ? 64 : (TMEM_NEED <= 128 ? 128 : (TMEM_NEED <= 256 ? 256 : 512));
  static constexpr uint32_t IDESC_ROW = tc_idesc(128, N, false);  // D1 += A X_J
  static constexpr uint32_t IDESC_COL = tc_idesc(128, N, true);   // D2 += A^T X_I (A read MN-major)
  static_assert(STAGE % 1024 == 0 && XB % 1024 == 0, "1024-byte swizzle alignment");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(TMEM_NEED <= 512, "tensor memory");
};

struct TsArgs {
  const uint8_t* tiles;  // packed tiles
  const uint8_t* xt;     // swizzled X^T tiles (NT x N*256 bytes)
  float* Y;              // padded, zero on entry
  const int* skip;
  Ctl* ctl;
  int rows;              // n * d
  int NT;
};

// Processing order: groups of R row tiles (I0 = g R), inside a group the
// columns J = I0 .. NT-1, inside a column ("strip") the rows I = I0 .. min(I0 +
// R, J + 1, NT) - 1.  Each tile appears once.  D1 (one slot per row of the
// group) lives across the group; D2 (the strip's column tile) across the strip.
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

template <int N>
__global__ void __launch_bounds__(192, 1) tc_sym_kernel(const TsArgs a) {
  using C = TsCfg<N>;
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
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(d1_empty + 1);
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = ts_tiles(a.NT);
  const long long t0 = total * blockIdx.x / gridDim.x;
  const long long t1 = total * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(xi_full, 1);
    mbar_init(xi_empty, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&d2_full[s], 1);
      mbar_init(&d2_empty[s], 4);
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
  const uint32_t tm_d1 = tmem;                      // + r * N
  const uint32_t tm_d2 = tmem + (uint32_t)(R * N);  // + db * N

  auto fail = [&]() {
    atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
    failed = 1;
  };

  if (t0 < t1 && warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int st = 0, p = 0;
    uint32_t ph = 0;
    long long it = 0;
    bool group_start = true;
    for (long long t = t0; t < t1 && !failed; ++t, ++it) {
      if (group_start) {  // X^T of the group's row tiles (one buffer: wait for the previous group)
        if (p >= 1 && !mbar_wait_bounded(xi_empty, (uint32_t)((p - 1) & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(xi_full, (uint32_t)(w.Rg * C::XB));
        bulk_g2s(smem + C::OFF_XI, a.xt + (long long)w.I0 * C::XB, (uint32_t)(w.Rg * C::XB), xi_full);
        ++p;
      }
      if (it >= C::NSTAGE && !mbar_wait_bounded(&empty[st], ph ^ 1u, kWaitLimitNs)) {
        fail();
        break;
      }
      uint8_t* stage = smem + st * C::STAGE;
      mbar_arrive_expect_tx(&full[st], C::STAGE);
      bulk_g2s(stage, a.tiles + t * (long long)kTsTileBytes, kTsTileBytes, &full[st]);
      bulk_g2s(stage + kTsTileBytes, a.xt + (long long)w.J * C::XB, C::XB, &full[st]);
      if (++st == C::NSTAGE) {
        st = 0;
        ph ^= 1u;
      }
      bool se, ge;
      w.next(se, ge);
      group_start = ge;
    }
    // Do not leave while copies into this CTA's shared memory may be in flight.
    const long long first = it > C::NSTAGE ? it - C::NSTAGE : 0;
    for (long long k = first; k < it; ++k)
      if (!mbar_wait_bounded(&full[k % C::NSTAGE], (uint32_t)((k / C::NSTAGE) & 1), kWaitLimitNs)) break;
    if (p >= 1) mbar_wait_bounded(xi_full, (uint32_t)((p - 1) & 1), kWaitLimitNs);
  } else if (t0 < t1 && warp == 1 && lane == 0) {
    // ------------------------------------------------------------- MMA issue
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int st = 0, p = 0;
    uint32_t ph = 0;
    long long k = 0;       // strips started
    bool group_start = true, strip_start = true;
    uint32_t started = 0;  // D1 slots written in this group segment
    for (long long t = t0; t < t1 && !failed; ++t) {
      if (group_start) {
        if (!mbar_wait_bounded(xi_full, (uint32_t)(p & 1), kWaitLimitNs) ||
            (p >= 1 && !mbar_wait_bounded(d1_empty, (uint32_t)((p - 1) & 1), kWaitLimitNs))) {
          fail();
          break;
        }
        started = 0;
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
      const int r = w.r;
      const uint32_t sa = smem_u32(smem + st * C::STAGE);
      const uint32_t sxj = sa + kTsTileBytes;
      const uint32_t sxi = smem_u32(smem + C::OFF_XI + r * C::XB);
      const bool first1 = !(started >> r & 1u);
      // D1[r] += A_IJ X_J: K = the tile's 128 columns, two 64-column halves of four K = 16 steps
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc_mma(tm_d1 + (uint32_t)(r * N), sw128_desc(sa + s * 1024 + kk * 32, 16, 2048),
                 sw128_desc(sxj + s * 1024 + kk * 32, 16, 2048), C::IDESC_ROW, (first1 && s == 0 && kk == 0) ? 0u : 1u);
      started |= 1u << r;
      // D2 += A_IJ^T X_I: K = the tile's 128 rows, eight K = 16 steps of two 8-row groups
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        tc_mma(tm_d2 + (uint32_t)(db * N), sw128_desc(sa + kk * 4096, 1024, 2048),
               sw128_desc(sxi + (kk >> 2) * 1024 + (kk & 3) * 32, 16, 2048), C::IDESC_COL,
               (strip_start && kk == 0) ? 0u : 1u);
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
        tc_commit(d1_full);
        tc_commit(xi_empty);
        ++p;
      }
      strip_start = se;
      group_start = ge;
    }
  } else if (t0 < t1 && warp >= 2) {
    // -------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31
    TsWalk<R> w;
    w.NT = a.NT;
    w.seek(t0);
    int p = 0;
    long long k = 0;
    uint32_t used = 0;  // D1 slots written in this group segment
    auto drain = [&](uint32_t taddr, int row) -> bool {  // TMEM rows 32q.. -> Y rows row.., then release
      float v[N];
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        float tt[16];
        tc_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, tt);
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c0 + c] = tt[c];
      }
      tc_wait_ld();
      if (row < a.rows) {
        float* y = a.Y + (long long)row * N;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 4) red_add_v4_f32(y + c0, v[c0], v[c0 + 1], v[c0 + 2], v[c0 + 3]);
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
        drain(tm_d2 + (uint32_t)(db * N), J * kTsTile + 32 * q + lane);
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
          if (used >> r & 1u) drain(tm_d1 + (uint32_t)(r * N), (I0 + r) * kTsTile + 32 * q + lane);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(d1_empty);
        used = 0;
        ++p;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_warp(tmem, (uint32_t)C::TMEM_COLS);
  }
}

// ------------------------------------------------------------ packing
// One CTA per tile (grid-stride): tile number t of the processing order, 2048
// 16-byte chunks of 8 consecutive columns.
template <int R, class Src>
__global__ void __launch_bounds__(256) ts_pack_kernel(Src src, int NT, uint8_t* out) {
  __shared__ int ij[2];
  const long long total = ts_tiles(NT);
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
    uint8_t* tile = out + t * (long long)kTsTileBytes;
    for (int ch = threadIdx.x; ch < kTsTile * kTsTile / 8; ch += blockDim.x) {
      const int r = ch >> 4, c = (ch & 15) * 8;
      const long long R = (long long)I * kTsTile + r, Cc = (long long)J * kTsTile + c;
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const __nv_bfloat16 lo = __float2bfloat16_rn(src(R, Cc + 2 * k));
        const __nv_bfloat16 hi = __float2bfloat16_rn(src(R, Cc + 2 * k + 1));
        w[k] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      }
      *reinterpret_cast<uint4*>(tile + ts_swz(r, c)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// X^T tiles: element (n, k) of tile J is X[128 J + k][n] in bfloat16 (zero past n*d rows).
__global__ void __launch_bounds__(256) ts_xt_kernel(const float* __restrict__ X, uint8_t* __restrict__ xt, int rows,
                                                   int D, int NT, const int* skip) {
  if (*skip) return;
  const long long chunks = (long long)NT * D * (kTsTile / 8);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < chunks;
       e += (long long)gridDim.x * blockDim.x) {
    const int J = (int)(e / (D * (kTsTile / 8)));
    const int rem = (int)(e % (D * (kTsTile / 8)));
    const int nn = rem / (kTsTile / 8), k0 = (rem % (kTsTile / 8)) * 8;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long r0 = (long long)J * kTsTile + k0 + 2 * k;
      const float a = r0 < rows ? X[r0 * D + nn] : 0.f;
      const float b = r0 + 1 < rows ? X[(r0 + 1) * D + nn] : 0.f;
      w[k] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
             ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
    }
    *reinterpret_cast<uint4*>(xt + (long long)J * D * 256 + ts_swz(nn, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------- host
bool tc_sym_supported(int d) { return d == 16 || d == 32 || d == 64; }

long long tc_sym_bytes(int n, int d) { return ts_tiles(ts_tile_rows(n, d)) * (long long)kTsTileBytes; }

// Bytes of the swizzled X^T tiles for (n, d).
long long tc_sym_xt_bytes(int n, int d) { return (long long)ts_tile_rows(n, d) * d * 256; }

template <int N>
static cudaError_t launch_ts(const TsArgs& a, cudaStream_t st, bool prepare) {
  using C = TsCfg<N>;
  if (prepare) return cudaFuncSetAttribute(tc_sym_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  const long long total = ts_tiles(a.NT);
  const int grid = (int)std::min<long long>(total, num_sms());
  tc_sym_kernel<N><<<grid, 192, C::SMEM, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_ts_any(int d, const TsArgs& a, cudaStream_t st, bool prepare) {
  switch (d) {
    case 16: return launch_ts<16>(a, st, prepare);
    case 32: return launch_ts<32>(a, st, prepare);
    case 64: return launch_ts<64>(a, st, prepare);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc_sym_prepare(int d) {
  TsArgs a{};
  return launch_ts_any(d, a, 0, true);
}

cudaError_t tc_sym_product(const void* packed, int n, int d, const float* X, uint8_t* xt, float* Y, Ctl* ctl,
                           const int* skip, cudaStream_t st) {
  const int NT = ts_tile_rows(n, d);
  const long long chunks = (long long)NT * d * (kTsTile / 8);
  const int g = (int)std::min<long long>((chunks + 255) / 256, 4LL * num_sms());
  ts_xt_kernel<<<g, 256, 0, st>>>(X, xt, n * d, d, NT, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TsArgs a{reinterpret_cast<const uint8_t*>(packed), xt, Y, skip, ctl, n * d, NT};
  return launch_ts_any(d, a, st, false);
}

template <class Src>
cudaError_t tc_sym_pack(Src src, int n, int d, void* packed, cudaStream_t st) {
  const int NT = ts_tile_rows(n, d);
  const int g = (int)std::min<long long>(ts_tiles(NT), 8LL * num_sms());
  uint8_t* out = reinterpret_cast<uint8_t*>(packed);
  switch (d) {
    case 16: ts_pack_kernel<TsCfg<16>::R><<<g, 256, 0, st>>>(src, NT, out); break;
    case 32: ts_pack_kernel<TsCfg<32>::R><<<g, 256, 0, st>>>(src, NT, out); break;
    case 64: ts_pack_kernel<TsCfg<64>::R><<<g, 256, 0, st>>>(src, NT, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t tc_sym_pack<UpperSrc>(UpperSrc, int, int, void*, cudaStream_t);
template cudaError_t tc_sym_pack<DenseSrc>(DenseSrc, int, int, void*, cudaStream_t);

}  // namespace nsrgs

// Y = A_off X on the CUDA cores in float32, reading only the upper triangle,
// for 8 < d <= 64 (NSRGS_F32 at these d): the symmetric read-once product of
// Algorithm 2's gradient where the d x d blocks are too wide for the
// register-resident panel stream.
//
// Layout ("float32 tile-upper"): the nd x nd matrix is cut into 64 x 64 tiles;
// tile (I, J) is stored for J >= I only, row after row of tiles (I = 0, 1, ..;
// J = I .. NT-1), 16 KB each.  A stored tile keeps the elements whose block row
// is above their block column (block(r) < block(c)); every other element
// (the block diagonal, blocks straddling the diagonal tile, the ragged edge)
// is zero, so every element of the strict block-upper triangle is stored once
// and the product needs no special case.  Inside a tile, rows are 256 bytes
// apart and 16-byte chunk k of row r sits at chunk k ^ ((r / 4) % 8), which
// keeps both of the kernel's shared-memory access patterns free of bank
// conflicts.  X enters as X^T tiles: for every 64-row tile J, DP x 64 floats
// (DP = d rounded up to a multiple of 8, the extra rows zero), element (c, k) =
// X[64 J + k][c].
//
// One stored tile feeds both products of the symmetric form:
//   Y_I += A_IJ X_J      (rows of tile I, summed over the tile's 64 columns)
//   Y_J += A_IJ^T X_I    (rows of tile J, summed over the tile's 64 rows).
// CTA (persistent over a contiguous range of the tile order; 9 warps):
//   warp 8 lane 0 : producer: cp.async.bulk of each tile and its X_J^T tile into
//                   a ring of stages, and of X_I^T into its own buffer when I
//                   changes; mbarrier expect_tx.
//   warps 0..3    : the row product.  Thread (p, cc, s) owns rows 4p .. 4p+3 of the
//                   tile, X columns 8cc .. 8cc+7 and the s-th of S column
//                   ranges; per 4 columns it reads 4 float4 of A and 8 float4 of
//                   X_J^T for 128 FMAs.  The row tile stays the same along a
//                   row of tiles, so the 32 partials stay in registers until I
//                   changes and are added to Y then.
//   warps 4..7    : the column product.  Thread (q, cc, s) owns tile columns
//                   4q .. 4q+3, X columns 8cc .. 8cc+7 and the s-th of S row
//                   ranges; per 4 rows it reads 4 float4 of A and 8 of X_I^T
//                   for 128 FMAs.  Its column tile changes with every tile: the
//                   S range partials are summed through shared memory and added
//                   to Y with red.global.add once per tile.
// S = 128 / (16 * DP/8) (8, 4, 2, 1 at DP = 8..64) keeps all 128 threads of a
// product busy.  Every wait is bounded; a timeout sets FLAG_TIMEOUT.
#include <algorithm>

#include "src.cuh"

namespace nsrgs {

constexpr int kFsT = 64;
constexpr int kFsTileBytes = kFsT * kFsT * 4;  // 16 KB

__host__ __device__ inline int fs_nt(int n, int d) { return (int)(((long long)n * d + kFsT - 1) / kFsT); }
__host__ __device__ inline long long fs_tiles(int NT) { return (long long)NT * (NT + 1) / 2; }
__host__ __device__ inline int fs_dp(int d) { return (d + 7) / 8 * 8; }
__host__ __device__ inline int fs_swz(int r, int c) { return r * 256 + (((c >> 2) ^ ((r >> 2) & 7)) << 4) + (c & 3) * 4; }
// first tile of row I in the order: I*NT - I*(I-1)/2
__host__ __device__ inline long long fs_row_start(int I, int NT) { return (long long)I * NT - (long long)I * (I - 1) / 2; }

// (I, J) of tile t of the processing order.
__host__ __device__ inline void fs_tile_ij(long long t, int NT, int& I, int& J) {
  const double b = 2.0 * NT + 1.0;
  int i = (int)((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (i < 0) i = 0;
  if (i > NT - 1) i = NT - 1;
  while (i > 0 && fs_row_start(i, NT) > t) --i;
  while (i + 1 < NT && fs_row_start(i + 1, NT) <= t) ++i;
  I = i;
  J = i + (int)(t - fs_row_start(i, NT));
}

template <int C>
struct FsCfg {
  static constexpr int DP = 8 * C;                  // X columns, padded to a multiple of 8
  static constexpr int S = C == 1 ? 8 : (C == 2 ? 4 : (C <= 4 ? 2 : 1));  // ranges per product
  static constexpr int TASKS = 16 * C * S;          // busy threads per product (<= 128)
  static constexpr int RANGE = kFsT / S;            // columns (rows) per range
  static constexpr int XB = DP * kFsT * 4;          // one X^T tile
  static constexpr int STAGE = kFsTileBytes + XB;   // A tile + X_J^T tile
  static constexpr int RED = S > 1 ? S * kFsT * DP * 4 : 0;  // column-product range partials
  // CTAs per SM: two (18 warps, 96 registers a thread) hide more latency for DP <= 32
  // (n = 2000: d = 16 1.29 -> 1.08 ms, d = 32 8.11 -> 7.40 ms); at DP = 64 the
  // 32-accumulator loop wants the registers of one CTA (48.7 vs 52.3 ms)
  static constexpr int MINB = C <= 4 ? 2 : 1;
  static constexpr int BUDGET = MINB == 2 ? 104 * 1024 : 200 * 1024;
  static constexpr int NSTAGE_RAW = (BUDGET - XB - RED) / STAGE;
  static constexpr int NSTAGE = NSTAGE_RAW > 8 ? 8 : NSTAGE_RAW;
  static constexpr int OFF_XI = NSTAGE * STAGE;
  static constexpr int OFF_RED = OFF_XI + XB;
  static constexpr int OFF_BARS = OFF_RED + RED;
  static constexpr int NBARS = 2 * NSTAGE + 4;
  static constexpr int SMEM = OFF_BARS + NBARS * 8;
  static constexpr int THREADS = 9 * 32;
  static_assert(TASKS <= 128, "tasks");
  static_assert(NSTAGE >= 2, "stages");
  static_assert(SMEM * MINB <= 227 * 1024, "shared memory");
};

struct FsArgs {
  const uint8_t* tiles;
  const float* xt;  // X^T tiles, NT x DP x 64 floats
  float* Y;         // padded, zero on entry
  const int* skip;
  Ctl* ctl;
  int rows;         // n * d
  int d;
  int NT;
};

template <int C>
__global__ void __launch_bounds__(FsCfg<C>::THREADS, FsCfg<C>::MINB) fs_sym_kernel(const __grid_constant__ FsArgs a) {
  using F = FsCfg<C>;
  constexpr int S = F::S, R = F::RANGE;
  if (*a.skip) return;  // uniform: written only by earlier launches
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + F::OFF_BARS);
  uint64_t* empty = full + F::NSTAGE;
  uint64_t* xi_full = empty + F::NSTAGE;
  uint64_t* xi_empty = xi_full + 1;
  uint64_t* rb_full = xi_empty + 1;  // column warps: every warp's range partials are written
  uint64_t* rb_free = rb_full + 1;   // column warps: every warp has read them
  float* red = reinterpret_cast<float*>(smem + F::OFF_RED);
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = fs_tiles(a.NT);
  const long long t0 = total * blockIdx.x / gridDim.x;
  const long long t1 = total * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < F::NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 8);
    }
    mbar_init(xi_full, 1);
    mbar_init(xi_empty, 4);
    mbar_init(rb_full, 4);
    mbar_init(rb_free, 4);
    failed = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (t0 >= t1) return;
  auto fail = [&]() {
    atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
    failed = 1;
  };

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int I, J;
      fs_tile_ij(t0, a.NT, I, J);
      int st = 0, p = 0;
      uint32_t ph = 0;
      long long it = 0;
      int Icur = -1;
      for (long long t = t0; t < t1 && !failed; ++t, ++it) {
        if (I != Icur) {  // X_I^T of the new row tile (one buffer: the column warps release the last)
          if (p >= 1 && !mbar_wait_bounded(xi_empty, (uint32_t)((p - 1) & 1), kWaitLimitNs)) {
            fail();
            break;
          }
          mbar_arrive_expect_tx(xi_full, (uint32_t)F::XB);
          bulk_g2s(smem + F::OFF_XI, a.xt + (long long)I * (F::XB / 4), (uint32_t)F::XB, xi_full);
          ++p;
          Icur = I;
        }
        if (it >= F::NSTAGE && !mbar_wait_bounded(&empty[st], ph ^ 1u, kWaitLimitNs)) {
          fail();
          break;
        }
        uint8_t* stage = smem + st * F::STAGE;
        mbar_arrive_expect_tx(&full[st], (uint32_t)F::STAGE);
        bulk_g2s(stage, a.tiles + t * (long long)kFsTileBytes, kFsTileBytes, &full[st]);
        bulk_g2s(stage + kFsTileBytes, a.xt + (long long)J * (F::XB / 4), (uint32_t)F::XB, &full[st]);
        if (++st == F::NSTAGE) {
          st = 0;
          ph ^= 1u;
        }
        if (++J == a.NT) {
          ++I;
          J = I;
        }
      }
      // Do not leave while copies into this CTA's shared memory may be in flight.
      const long long first = it > F::NSTAGE ? it - F::NSTAGE : 0;
      for (long long k = first; k < it; ++k)
        if (!mbar_wait_bounded(&full[k % F::NSTAGE], (uint32_t)((k / F::NSTAGE) & 1), kWaitLimitNs)) break;
      if (p >= 1) mbar_wait_bounded(xi_full, (uint32_t)((p - 1) & 1), kWaitLimitNs);
    }
    return;
  }

  const bool rowp = warp < 4;  // row product (warps 0-3) or column product (warps 4-7)
  const int u = threadIdx.x & 127;
  const bool busy = u < F::TASKS;
  const int g = u & 15;          // row group p (row product) / column group q (column product)
  const int cs = u >> 4;
  const int cc = cs % C;         // X columns 8cc .. 8cc+7
  const int s = cs / C;          // range
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[i][c] = 0.f;
  const bool vec_y = (a.d & 3) == 0;
  // add acc (rows row0 .. row0+3 of Y, X columns 8cc ..) to Y
  auto flush = [&](int row0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = row0 + i;
      if (row >= a.rows) continue;
      float* y = a.Y + (long long)row * a.d + 8 * cc;
      if (vec_y && 8 * cc + 8 <= a.d) {
        red_add_v4_f32(y, acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        red_add_v4_f32(y + 4, acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (8 * cc + c < a.d) red_add_f32(y + c, acc[i][c]);
      }
    }
  };

  int I, J;
  fs_tile_ij(t0, a.NT, I, J);
  int st = 0, p = 0;
  uint32_t ph = 0;
  int Icur = -1;
  long long kt = 0;  // tiles done by this thread's warp
  for (long long t = t0; t < t1; ++t, ++kt) {
    if (failed) break;
    if (!rowp && I != Icur) {
      if (p >= 1) {  // done with the previous X_I^T
        __syncwarp();
        if (lane == 0) mbar_arrive(xi_empty);
      }
      if (!mbar_wait_bounded(xi_full, (uint32_t)(p & 1), kWaitLimitNs)) {
        fail();
        break;
      }
      ++p;
    }
    if (rowp && I != Icur && Icur >= 0) {
      if (busy) flush(Icur * kFsT + 4 * g);  // the finished row tile's partials (one per range)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[i][c] = 0.f;
    }
    Icur = I;
    if (!mbar_wait_bounded(&full[st], ph, kWaitLimitNs)) {
      fail();
      break;
    }
    const uint8_t* A = smem + st * F::STAGE;
    if (rowp) {
      const float* XJ = reinterpret_cast<const float*>(A + kFsTileBytes) + (8 * cc) * kFsT;
      if (busy) {
#pragma unroll(F::MINB == 2 ? 2 : 4)
        for (int k = s * R; k < (s + 1) * R; k += 4) {
          float4 av[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4*>(A + fs_swz(4 * g + i, k));
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 x = *reinterpret_cast<const float4*>(XJ + c * kFsT + k);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float v = acc[i][c];
              v = fmaf(av[i].x, x.x, v);
              v = fmaf(av[i].y, x.y, v);
              v = fmaf(av[i].z, x.z, v);
              v = fmaf(av[i].w, x.w, v);
              acc[i][c] = v;
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    } else {
      const float* XI = reinterpret_cast<const float*>(smem + F::OFF_XI) + (8 * cc) * kFsT;
      if (busy) {
#pragma unroll(F::MINB == 2 ? 2 : 4)
        for (int r = s * R; r < (s + 1) * R; r += 4) {
          float4 av[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4*>(A + fs_swz(r + i, 4 * g));
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 x = *reinterpret_cast<const float4*>(XI + c * kFsT + r);
            acc[0][c] = fmaf(av[0].x, x.x, fmaf(av[1].x, x.y, fmaf(av[2].x, x.z, fmaf(av[3].x, x.w, acc[0][c]))));
            acc[1][c] = fmaf(av[0].y, x.x, fmaf(av[1].y, x.y, fmaf(av[2].y, x.z, fmaf(av[3].y, x.w, acc[1][c]))));
            acc[2][c] = fmaf(av[0].z, x.x, fmaf(av[1].z, x.y, fmaf(av[2].z, x.z, fmaf(av[3].z, x.w, acc[2][c]))));
            acc[3][c] = fmaf(av[0].w, x.x, fmaf(av[1].w, x.y, fmaf(av[2].w, x.z, fmaf(av[3].w, x.w, acc[3][c]))));
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);  // the stage is read; the flush below uses registers
      if constexpr (S == 1) {
        if (busy) flush(J * kFsT + 4 * g);
      } else {
        // sum the S range partials of each (column, X column) through shared memory;
        // the four column warps meet on mbarriers (bounded waits), not bar.sync
        if (kt >= 1 && !mbar_wait_bounded(rb_free, (uint32_t)((kt - 1) & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        // scratch order [range][X column][tile column]: a thread's 4 columns are one
        // float4, and the 8 threads of a quarter-warp write 8 consecutive float4s
        if (busy) {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            *reinterpret_cast<float4*>(red + ((s * F::DP + 8 * cc + c) * kFsT + 4 * g)) =
                make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(rb_full);
        if (!mbar_wait_bounded(rb_full, (uint32_t)(kt & 1), kWaitLimitNs)) {
          fail();
          break;
        }
        // 64 columns x DP values, 4 consecutive X columns per thread and pass (one
        // float4 of Y): sum over the ranges, add to Y; consecutive threads take
        // consecutive tile columns, so the scratch reads are conflict-free
        for (int e = u; e < kFsT * (F::DP / 4); e += 128) {
          const int col = e % kFsT, xc = (e / kFsT) * 4;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int r2 = 0; r2 < S; ++r2) {
            const float* w = red + (r2 * F::DP + xc) * kFsT + col;
            v.x += w[0];
            v.y += w[kFsT];
            v.z += w[2 * kFsT];
            v.w += w[3 * kFsT];
          }
          const int row = J * kFsT + col;
          if (row < a.rows && xc < a.d) {
            float* y = a.Y + (long long)row * a.d + xc;
            if (vec_y) {
              red_add_v4_f32(y, v.x, v.y, v.z, v.w);
            } else {
              red_add_f32(y, v.x);
              if (xc + 1 < a.d) red_add_f32(y + 1, v.y);
              if (xc + 2 < a.d) red_add_f32(y + 2, v.z);
              if (xc + 3 < a.d) red_add_f32(y + 3, v.w);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(rb_free);  // read: the next tile may overwrite them
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[i][c] = 0.f;
    }
    if (++st == F::NSTAGE) {
      st = 0;
      ph ^= 1u;
    }
    if (++J == a.NT) {
      ++I;
      J = I;
    }
  }
  if (rowp && busy && Icur >= 0 && !failed) flush(Icur * kFsT + 4 * g);
}

// ------------------------------------------------------------ packing
// One CTA per tile (grid-stride): element (r, c) of tile t of the order is the
// stored element (block(row) < block(col)) or zero; 1024 16-byte chunks per tile.
template <class Src>
__global__ void __launch_bounds__(256) fs_pack_kernel(Src src, int NT, int d, uint8_t* out) {
  const long long total = fs_tiles(NT);
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    int I, J;
    fs_tile_ij(t, NT, I, J);
    uint8_t* tile = out + t * (long long)kFsTileBytes;
    for (int ch = threadIdx.x; ch < kFsT * kFsT / 4; ch += blockDim.x) {
      const int r = ch >> 4, c = (ch & 15) * 4;
      const long long R = (long long)I * kFsT + r, Cc = (long long)J * kFsT + c;
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = src(R, Cc + k);  // zero on and below the block diagonal, and outside
      *reinterpret_cast<float4*>(tile + fs_swz(r, c)) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// X^T tiles: element (c, k) of tile J is X[64 J + k][c] (zero past n*d rows and for c >= d).
__global__ void __launch_bounds__(256) fs_xt_kernel(const float* __restrict__ X, float* __restrict__ xt, int rows,
                                                   int d, int DP, int NT, const int* skip) {
  if (*skip) return;
  const long long count = (long long)NT * DP * kFsT;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % kFsT);
    const long long rest = e / kFsT;
    const int c = (int)(rest % DP);
    const int J = (int)(rest / DP);
    const long long row = (long long)J * kFsT + k;
    xt[e] = (c < d && row < rows) ? X[row * d + c] : 0.f;
  }
}

// ---------------------------------------------------------------- host
bool fs_sym_supported(int d) { return d > 8 && d <= 64; }
long long fs_sym_bytes(int n, int d) { return fs_tiles(fs_nt(n, d)) * (long long)kFsTileBytes; }
long long fs_sym_xt_bytes(int n, int d) { return (long long)fs_nt(n, d) * fs_dp(d) * kFsT * 4; }

template <int C>
static cudaError_t launch_fs(const FsArgs& a, cudaStream_t st, bool prepare) {
  using F = FsCfg<C>;
  if (prepare) return cudaFuncSetAttribute(fs_sym_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM);
  const long long total = fs_tiles(a.NT);
  const int grid = (int)std::min<long long>(total, (long long)F::MINB * num_sms());
  fs_sym_kernel<C><<<grid, F::THREADS, F::SMEM, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_fs_any(int d, const FsArgs& a, cudaStream_t st, bool prepare) {
  switch (fs_dp(d) / 8) {
    case 2: return launch_fs<2>(a, st, prepare);
    case 3: return launch_fs<3>(a, st, prepare);
    case 4: return launch_fs<4>(a, st, prepare);
    case 5: return launch_fs<5>(a, st, prepare);
    case 6: return launch_fs<6>(a, st, prepare);
    case 7: return launch_fs<7>(a, st, prepare);
    case 8: return launch_fs<8>(a, st, prepare);
  }
  return cudaErrorInvalidValue;
}

cudaError_t fs_sym_prepare(int d) {
  FsArgs a{};
  return launch_fs_any(d, a, 0, true);
}

// Y = A_off X for A packed with block size d and X of `width` columns (width = d
// in Algorithm 2; the Stiefel form's p >= d): the tiles hold elements, so only
// the number of rows (n d) and the width of X enter the product.
cudaError_t fs_sym_product_w(const void* packed, int n, int d, int width, const float* X, float* xt, float* Y,
                             Ctl* ctl, const int* skip, cudaStream_t st) {
  const int NT = fs_nt(n, d);
  const int DP = fs_dp(width);
  const long long count = (long long)NT * DP * kFsT;
  const int g = (int)std::min<long long>((count + 255) / 256, 4LL * num_sms());
  fs_xt_kernel<<<g, 256, 0, st>>>(X, xt, n * d, width, DP, NT, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  FsArgs a{reinterpret_cast<const uint8_t*>(packed), xt, Y, skip, ctl, n * d, width, NT};
  return launch_fs_any(width, a, st, false);
}

cudaError_t fs_sym_product(const void* packed, int n, int d, const float* X, float* xt, float* Y, Ctl* ctl,
                           const int* skip, cudaStream_t st) {
  return fs_sym_product_w(packed, n, d, d, X, xt, Y, ctl, skip, st);
}

// Bytes of the X^T tiles of fs_sym_product_w.
long long fs_sym_xt_bytes_w(int n, int d, int width) { return (long long)fs_nt(n, d) * fs_dp(width) * kFsT * 4; }

template <class Src>
cudaError_t fs_sym_pack(Src src, int n, int d, void* packed, cudaStream_t st) {
  const int NT = fs_nt(n, d);
  const int g = (int)std::min<long long>(fs_tiles(NT), 8LL * num_sms());
  fs_pack_kernel<<<g, 256, 0, st>>>(src, NT, d, reinterpret_cast<uint8_t*>(packed));
  return cudaGetLastError();
}
template cudaError_t fs_sym_pack<UpperSrc>(UpperSrc, int, int, void*, cudaStream_t);
template cudaError_t fs_sym_pack<DenseSrc>(DenseSrc, int, int, void*, cudaStream_t);
template cudaError_t fs_sym_pack<SeAugSrc>(SeAugSrc, int, int, void*, cudaStream_t);

}  // namespace nsrgs

// Y = A_off X on the 5th-generation tensor cores (tcgen05) for block sizes
// d in {16, 32, 64}, with A stored densely in bfloat16 (NSRGS_DENSE_BF16) and
// X rounded to bfloat16 each launch; products accumulate in float32 in TMEM.
//
// Per CTA (6 warps, persistent over work units = 128-row tile x K chunk):
//   warp 0 lane 0 : TMA producer.  cp.async.bulk.tensor 2-D loads of the A tile
//                   (128 rows x 64 columns, 128-byte swizzle) and of the X^T tile
//                   (d rows x 64 columns) into a ring of shared-memory stages,
//                   completion on mbarriers (expect_tx).
//   warp 1        : allocates / frees TMEM (d fp32 columns x 128 lanes); lane 0
//                   issues tcgen05.mma (M = 128, N = d, K = 16) four times per
//                   stage and tcgen05.commit's the stage back to the producer
//                   and, after a unit's last stage, the accumulator to the epilogue.
//   warps 2..5    : epilogue.  tcgen05.ld the 128 x d accumulator (each warp its
//                   32-lane quarter), release it, add the rows to Y with
//                   red.global.add.v4.f32 (units split K, so rows are summed).
// This is the dense form (both triangles, no symmetric reuse): for d >= 16 the
// product is a tall-skinny GEMM that the tensor cores finish at HBM speed.
// Every wait is bounded; a timeout sets FLAG_TIMEOUT, the CTA still reaches
// its final barrier and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <string>

#include "tc_common.cuh"

namespace nsrgs {

template <int N>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int BK = 64;                       // 64 bf16 = one 128-byte swizzle row
  static constexpr int A_BYTES = BM * BK * 2;         // 16 KB
  static constexpr int B_BYTES = N * BK * 2;          // 2, 4 or 8 KB
  static constexpr int STAGE = A_BYTES + B_BYTES;     // multiple of 1024 (swizzle atoms)
  static constexpr int NSTAGE = 6;
  static constexpr int TMEM_COLS = N < 32 ? 32 : N;   // power of two >= 32
  static constexpr int OFF_BARS = NSTAGE * STAGE;
  static constexpr int SMEM = 1024 + OFF_BARS + (2 * NSTAGE + 2) * 8 + 16;
  static constexpr uint32_t IDESC = tc_idesc(BM, N, false);  // both operands K-major
  static_assert(STAGE % 1024 == 0, "stages must keep 1024-byte swizzle alignment");
};

struct TcArgs {
  float* Y;        // padded, zero on entry
  const int* skip;
  Ctl* ctl;
  int rows;        // n * d
  int row_tiles;   // ceil(rows / 128)
  int ksteps;      // pitch / 64
  int splits;      // K chunks per row tile
};

__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int N>
__global__ void __launch_bounds__(192, 1)
    tc_dense_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
  using C = TcCfg<N>;
  if (*a.skip) return;  // uniform: written only by earlier launches
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::OFF_BARS);
  uint64_t* empty = full + C::NSTAGE;
  uint64_t* acc_full = empty + C::NSTAGE;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = a.row_tiles * a.splits;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4);
    failed = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc_warp(tmem_slot, (uint32_t)C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    int it = 0, st = 0;
    uint32_t ph = 0;
    for (int u = blockIdx.x; u < units && !failed; u += gridDim.x) {
      const int m = u / a.splits, c = u % a.splits;
      const int kb = (int)((long long)c * a.ksteps / a.splits), ke = (int)((long long)(c + 1) * a.ksteps / a.splits);
      for (int ks = kb; ks < ke; ++ks, ++it) {
        if (it >= C::NSTAGE && !mbar_wait_bounded(&empty[st], ph ^ 1u, kWaitLimitNs)) {
          atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
          failed = 1;
          break;
        }
        uint8_t* stage = smem + st * C::STAGE;
        mbar_arrive_expect_tx(&full[st], C::STAGE);
        tma_load_2d(stage, &tmA, ks * C::BK, m * C::BM, &full[st]);
        tma_load_2d(stage + C::A_BYTES, &tmB, ks * C::BK, 0, &full[st]);
        if (++st == C::NSTAGE) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------- MMA issue
    int st = 0, j = 0;
    uint32_t ph = 0;
    for (int u = blockIdx.x; u < units && !failed; u += gridDim.x, ++j) {
      const int c = u % a.splits;
      const int kb = (int)((long long)c * a.ksteps / a.splits), ke = (int)((long long)(c + 1) * a.ksteps / a.splits);
      if (j > 0 && !mbar_wait_bounded(acc_empty, (uint32_t)((j - 1) & 1), kWaitLimitNs)) {
        atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
        failed = 1;
        break;
      }
      tc_fence_after();
      for (int ks = kb; ks < ke; ++ks) {
        if (!mbar_wait_bounded(&full[st], ph, kWaitLimitNs)) {
          atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
          failed = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * C::STAGE);
        const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
        for (int kk = 0; kk < C::BK / 16; ++kk)
          tc_mma(tmem, sw128_desc(sa + kk * 32, 16, 1024), sw128_desc(sb + kk * 32, 16, 1024), C::IDESC, (ks > kb || kk > 0) ? 1u : 0u);
        tc_commit(&empty[st]);
        if (++st == C::NSTAGE) {
          st = 0;
          ph ^= 1u;
        }
      }
      tc_commit(acc_full);
    }
  } else if (warp >= 2) {
    // -------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31
    int j = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
      if (!mbar_wait_bounded(acc_full, (uint32_t)(j & 1), kWaitLimitNs)) {
        atomicOr(&a.ctl->flags, FLAG_TIMEOUT);
        failed = 1;
        break;
      }
      tc_fence_after();
      float v[N];
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        float t[16];
        tc_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, t);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[c0 + k] = t[k];
      }
      tc_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      const int row = (u / a.splits) * C::BM + 32 * q + lane;
      if (row < a.rows) {
        float* y = a.Y + (long long)row * N;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 4) red_add_v4_f32(y + c0, v[c0], v[c0 + 1], v[c0 + 2], v[c0 + 3]);
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

// X^T in bfloat16: XT[c][r] = X[r][c] for r < rows, zero up to the pitch.
__global__ void xt_bf16_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ XT, int rows, int D, int pitch,
                               const int* skip) {
  if (*skip) return;
  const long long total = (long long)D * pitch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / pitch), r = (int)(e % pitch);
    XT[e] = __float2bfloat16_rn(r < rows ? X[(long long)r * D + c] : 0.f);
  }
}

// ---------------------------------------------------------------- host
long long dense_bf16_pitch(int n, int d) { return ((long long)n * d + 63) / 64 * 64; }

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

static bool make_map(CUtensorMap* tm, const void* base, uint64_t cols, uint64_t rows, uint64_t pitch_bytes,
                     uint32_t box_cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N>
static cudaError_t launch_tc(const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a, cudaStream_t st,
                             bool prepare) {
  using C = TcCfg<N>;
  if (prepare)
    return cudaFuncSetAttribute(tc_dense_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  const int units = a.row_tiles * a.splits;
  const int grid = units < num_sms() ? units : num_sms();
  tc_dense_kernel<N><<<grid, 192, C::SMEM, st>>>(ta, tb, a);
  return cudaGetLastError();
}

bool tc_dense_supported(int d) { return d == 16 || d == 32 || d == 64; }

cudaError_t tc_dense_prepare(int d) {
  CUtensorMap dummy;
  TcArgs a{};
  switch (d) {
    case 16: return launch_tc<16>(dummy, dummy, a, 0, true);
    case 32: return launch_tc<32>(dummy, dummy, a, 0, true);
    case 64: return launch_tc<64>(dummy, dummy, a, 0, true);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ autotuner
// Split-K (K chunks per 128-row tile) per (n, d): the first call for a shape made
// outside any stream capture times a few candidates and keeps the fastest; until
// then (and inside captures) the heuristic of about two work units per SM is used.
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tuned_splits;

static int heuristic_splits(int row_tiles, int ksteps) {
  int s = (2 * num_sms() + row_tiles - 1) / row_tiles;
  if (s < 1) s = 1;
  if (s > ksteps) s = ksteps;
  return s;
}

static cudaError_t launch_tc_any(int d, const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a,
                                 cudaStream_t st) {
  switch (d) {
    case 16: return launch_tc<16>(ta, tb, a, st, false);
    case 32: return launch_tc<32>(ta, tb, a, st, false);
    case 64: return launch_tc<64>(ta, tb, a, st, false);
  }
  return cudaErrorInvalidValue;
}

static bool build_launch(const void* packed, int n, int d, __nv_bfloat16* XT, float* Y, Ctl* ctl, const int* skip,
                         CUtensorMap* ta, CUtensorMap* tb, TcArgs* a) {
  const int rows = n * d;
  const long long pitch = dense_bf16_pitch(n, d);
  if (!make_map(ta, packed, (uint64_t)pitch, (uint64_t)rows, (uint64_t)pitch * 2, 64, 128) ||
      !make_map(tb, XT, (uint64_t)pitch, (uint64_t)d, (uint64_t)pitch * 2, 64, (uint32_t)d))
    return false;
  a->Y = Y;
  a->skip = skip;
  a->ctl = ctl;
  a->rows = rows;
  a->row_tiles = (rows + 127) / 128;
  a->ksteps = (int)(pitch / 64);
  a->splits = heuristic_splits(a->row_tiles, a->ksteps);
  return true;
}

// Times candidate splits with the caller's buffers (Y is left with garbage: the
// caller clears it before use).  No-op when the shape is already tuned or `st`
// is capturing.
cudaError_t tc_dense_tune(const void* packed, int n, int d, __nv_bfloat16* XT, float* Y, Ctl* ctl, const int* skip,
                          cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tuned_splits.count({n, d})) return cudaSuccess;
  }
  cudaStreamCaptureStatus cs;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
  CUtensorMap ta, tb;
  TcArgs a;
  if (!build_launch(packed, n, d, XT, Y, ctl, skip, &ta, &tb, &a)) return cudaErrorInvalidValue;
  const int base = heuristic_splits(a.row_tiles, a.ksteps);
  int best = base;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
  const int cands[5] = {base / 2, base, 2 * base, 4 * base, 8 * base};
  for (int c : cands) {
    if (c < 1 || c > a.ksteps) continue;
    a.splits = c;
    if ((e = launch_tc_any(d, ta, tb, a, st)) != cudaSuccess) break;  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r)
      if ((e = launch_tc_any(d, ta, tb, a, st)) != cudaSuccess) break;
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_splits[{n, d}] = best;
  return cudaSuccess;
}

int tc_dense_splits(int n, int d) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_splits.find({n, d});
  return it == g_tuned_splits.end() ? 0 : it->second;
}

// XT: workspace buffer of d * pitch bf16.
cudaError_t tc_dense_product(const void* packed, int n, int d, const float* X, __nv_bfloat16* XT, float* Y, Ctl* ctl,
                             const int* skip, cudaStream_t st) {
  const int rows = n * d;
  const long long pitch = dense_bf16_pitch(n, d);
  xt_bf16_kernel<<<2 * num_sms(), 256, 0, st>>>(X, XT, rows, d, (int)pitch, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap ta, tb;
  TcArgs a;
  if (!build_launch(packed, n, d, XT, Y, ctl, skip, &ta, &tb, &a)) return cudaErrorInvalidValue;
  const int tuned = tc_dense_splits(n, d);
  if (tuned > 0) a.splits = tuned;
  return launch_tc_any(d, ta, tb, a, st);
}

}  // namespace nsrgs

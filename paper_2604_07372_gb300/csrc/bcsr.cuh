// Block-sparse rows (NSRGS_BCSR_F32 / NSRGS_BCSR_BF16): layout helpers and the
// warp-per-row product Y_i = sum_j A_ij X_j shared by the single-instance and
// the batched streams.  The layout is described in bcsr.cu.
#pragma once

#include "common.cuh"

namespace nsrgs {

constexpr int kBcsrHeader = 64;

__host__ __device__ inline long long bcsr_align(long long x) { return (x + 15) / 16 * 16; }
__host__ __device__ inline int bcsr_elem_bytes(int storage) { return storage == NSRGS_BCSR_BF16 ? 2 : 4; }
__host__ __device__ inline long long bcsr_off_col(int n) { return bcsr_align(kBcsrHeader + 8LL * (n + 1)); }
__host__ __device__ inline long long bcsr_off_val(int n, long long nnzb) {
  return bcsr_align(bcsr_off_col(n) + 4LL * nnzb);
}
__host__ __device__ inline long long bcsr_bytes_of(int n, int d, int storage, long long nnzb) {
  const long long b = bcsr_off_val(n, nnzb) + nnzb * d * d * bcsr_elem_bytes(storage);
  return (b + 255) / 256 * 256;
}
long long bcsr_bytes(int n, int d, int storage, long long nnzb);

__device__ __forceinline__ float bcsr_load(const float* p) { return __ldg(p); }
__device__ __forceinline__ float bcsr_load(const __nv_bfloat16* p) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
}

// Lanes per block for d <= 5: d*d lanes work on one block, lane (m, c) owning
// X_j[m][c] and column m of A_ij, so a gather of X_j touches the block's own
// 4 d^2 bytes once instead of once per lane and element; 32 / (d*d) blocks per
// warp step.  Partials acc[r] (the lane's share of Y_i[r][c]) are summed per
// (r, c) through a warp-private shared-memory scratch of 32 d floats, in lane
// order (deterministic), and Y_i is stored.
template <int D, class T>
__device__ __forceinline__ void bcsr_row_product_lanes(const uint8_t* __restrict__ packed, long long i,
                                                       const float* __restrict__ X, float* __restrict__ Y, int lane,
                                                       float* red) {
  constexpr int LPB = D * D, BPW = 32 / LPB, U = 16;  // 16 blocks per lane group in flight
  const long long* hdr = reinterpret_cast<const long long*>(packed);
  const long long* rowptr = reinterpret_cast<const long long*>(packed + kBcsrHeader);
  const int* col = reinterpret_cast<const int*>(packed + hdr[3]);
  const T* val = reinterpret_cast<const T*>(packed + hdr[4]);
  const int slot = lane / LPB, e = lane % LPB, m = e / D, c = e % D;
  const bool on = slot < BPW;
  float acc[D];
#pragma unroll
  for (int r = 0; r < D; ++r) acc[r] = 0.f;
  const long long k1 = rowptr[i + 1];
  for (long long k0 = rowptr[i]; k0 < k1; k0 += BPW * U) {
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long k = k0 + u * BPW + slot;
      j[u] = (on && k < k1) ? __ldg(col + k) : -1;
    }
    float xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = j[u] >= 0 ? __ldg(X + (long long)j[u] * LPB + m * D + c) : 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j[u] < 0) continue;
      const T* a = val + (k0 + u * BPW + slot) * LPB;
#pragma unroll
      for (int r = 0; r < D; ++r) acc[r] = fmaf(bcsr_load(a + r * D + m), xv[u], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < D; ++r) red[lane * D + r] = on ? acc[r] : 0.f;
  __syncwarp();
  if (lane < LPB) {
    const int rr = lane / D, cc = lane % D;
    float v = 0.f;
    for (int l = 0; l < BPW * LPB; ++l)
      if ((l % LPB) % D == cc) v += red[l * D + rr];
    Y[i * LPB + lane] = v;
  }
  __syncwarp();
}

// One warp: Y_i = sum_j A_ij X_j for block row i of the packed buffer.  For
// d <= 5 see bcsr_row_product_lanes.  Above, lanes take the row's blocks in
// turn (U per pass, their column and value loads issued together so the
// dependent X_j gathers overlap), accumulate d x d partials in registers one
// X_j row at a time, then a warp reduction; Y_i is written, not accumulated.
// `red`: warp-private shared scratch of at least 32 * 5 floats.
template <int D, class T>
__device__ __forceinline__ void bcsr_row_product(const uint8_t* __restrict__ packed, long long i,
                                                 const float* __restrict__ X, float* __restrict__ Y, int lane,
                                                 float* red) {
  if constexpr (D <= 5) {
    bcsr_row_product_lanes<D, T>(packed, i, X, Y, lane, red);
    return;
  }
  const long long* hdr = reinterpret_cast<const long long*>(packed);
  const long long* rowptr = reinterpret_cast<const long long*>(packed + kBcsrHeader);
  const int* col = reinterpret_cast<const int*>(packed + hdr[3]);
  const T* val = reinterpret_cast<const T*>(packed + hdr[4]);
  float acc[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) acc[r][c] = 0.f;
  constexpr int U = D <= 4 ? 4 : (D <= 6 ? 2 : 1);
  const long long k1 = rowptr[i + 1];
  for (long long k = rowptr[i] + lane; k < k1; k += 32 * U) {
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = (k + 32 * u < k1) ? __ldg(col + k + 32 * u) : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j[u] < 0) continue;
      const T* a = val + (k + 32 * u) * D * D;
      const float* x = X + (long long)j[u] * D * D;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        float xr[D], am[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xr[c] = __ldg(x + m * D + c);
#pragma unroll
        for (int r = 0; r < D; ++r) am[r] = bcsr_load(a + r * D + m);
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) acc[r][c] = fmaf(am[r], xr[c], acc[r][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float v = acc[r][c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[r][c] = v;
    }
  float* y = Y + i * D * D;
  for (int e = lane; e < D * D; e += 32) {
    float v = 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (r * D + c == e) v = acc[r][c];
    y[e] = v;
  }
}

}  // namespace nsrgs

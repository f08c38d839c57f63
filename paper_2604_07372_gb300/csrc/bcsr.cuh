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

// One warp: Y_i = sum_j A_ij X_j for block row i of the packed buffer.  Lanes
// take the row's blocks in turn (U per pass, their column and value loads
// issued together so the dependent X_j gathers overlap), accumulate d x d
// partials in registers one X_j row at a time, then a warp reduction; Y_i is
// written, not accumulated.  (A mapping with d*d lanes per block, which reads
// each X_j once per block instead of once per element, measured slower.)
template <int D, class T>
__device__ __forceinline__ void bcsr_row_product(const uint8_t* __restrict__ packed, long long i,
                                                 const float* __restrict__ X, float* __restrict__ Y, int lane) {
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

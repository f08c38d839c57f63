// Block-sparse rows (NSRGS_BCSR_F32 / NSRGS_BCSR_BF16): layout helpers and the
// warp-per-row product Y_i = sum_j A_ij X_j shared by the single-instance and
// the batched streams.  The layout is described in bcsr.cu.
#pragma once

#include "common.cuh"

namespace nsrgs {

constexpr int kBcsrHeader = 64;
constexpr int kBcsrWarps = 4;  // warps per CTA of the row kernels

__host__ __device__ inline long long bcsr_align(long long x) { return (x + 15) / 16 * 16; }
__host__ __device__ inline int bcsr_elem_bytes(int storage) { return storage == NSRGS_BCSR_BF16 ? 2 : 4; }
__host__ __device__ inline long long bcsr_off_col(int n) { return bcsr_align(kBcsrHeader + 8LL * (n + 1)); }
__host__ __device__ inline long long bcsr_off_val(int n, long long nnzb) {
  return bcsr_align(bcsr_off_col(n) + 4LL * nnzb);
}
// Blocks are stored in groups of 32 (the last group padded with zeros).
__host__ __device__ inline long long bcsr_val_slots(long long nnzb) { return (nnzb + 31) / 32 * 32; }
// Element e (= r*d + c) of stored block k: the 32 blocks of a group are
// interleaved element by element, so the 32 lanes of a warp that take blocks
// k0 .. k0+31 read element e of all of them from one or two 128-byte lines.
__host__ __device__ inline long long bcsr_val_pos(long long k, int e, int dd) {
  return (k >> 5) * 32LL * dd + (long long)e * 32 + (k & 31);
}
__host__ __device__ inline long long bcsr_bytes_of(int n, int d, int storage, long long nnzb) {
  const long long b = bcsr_off_val(n, nnzb) + bcsr_val_slots(nnzb) * d * d * bcsr_elem_bytes(storage);
  return (b + 255) / 256 * 256;
}
long long bcsr_bytes(int n, int d, int storage, long long nnzb);

__device__ __forceinline__ float bcsr_load(const float* p) { return __ldg(p); }
__device__ __forceinline__ float bcsr_load(const __nv_bfloat16* p) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
}

// X_j (d x d, row-major at j*d*d) is 16-byte aligned for even d and is then
// read with 128-bit loads; for odd d >= 3 the warp gathers the 32 X_j of a pass
// together through shared memory (element f of the pass's 32*d*d values by lane
// f mod 32), so that one load instruction touches a few lines instead of 32.
template <int D>
struct BcsrX {
  static constexpr int DD = D * D;
  static constexpr bool kCoop = (D % 2 == 1) && D >= 3;
  // passes of 32 blocks per loop trip (their loads are in flight together)
  static constexpr int kU = D <= 2 ? 4 : (D <= 4 ? 2 : 1);
  static constexpr int kSmemFloats = kCoop ? kU * 32 * DD : 1;  // per warp
};

// One warp: Y_i = sum_j A_ij X_j for block row i of the packed buffer.  Lane l
// takes blocks rowptr[i] + l, + 32 + l, ...; per loop trip it loads the column
// indices and d*d values of kU such blocks (coalesced by the interleaved
// layout), gathers their X_j, and accumulates the d x d partial in registers; a
// warp reduction ends the row, and Y_i is written, not accumulated.  xs: this
// warp's shared-memory buffer of BcsrX<D>::kSmemFloats floats (odd d >= 3).
// A row range outside the stored blocks or a misaligned X for the vector loads
// is flagged (FLAG_BAD_LAYOUT in ctl) and the row skipped; a column index is
// clamped into [0, n).  A corrupted buffer thus cannot fault the device.
template <int D, class T>
__device__ __forceinline__ void bcsr_row_product(const uint8_t* __restrict__ packed, long long i,
                                                 const float* __restrict__ X, float* __restrict__ Y, int lane,
                                                 float* xs, Ctl* ctl) {
  constexpr int DD = D * D;
  constexpr int U = BcsrX<D>::kU;
  const long long* hdr = reinterpret_cast<const long long*>(packed);
  const long long* rowptr = reinterpret_cast<const long long*>(packed + kBcsrHeader);
  const int* col = reinterpret_cast<const int*>(packed + hdr[3]);
  const T* val = reinterpret_cast<const T*>(packed + hdr[4]);
  const long long n = hdr[0], nnzb = hdr[2];
  const long long k0 = rowptr[i], k1 = rowptr[i + 1];
  constexpr bool kVecX = !BcsrX<D>::kCoop && DD % 4 == 0;
  if (n < 1 || k0 < 0 || k1 < k0 || k1 > nnzb || (kVecX && (reinterpret_cast<uintptr_t>(X) & 15u))) {
    if (lane == 0) atomicOr(&ctl->flags, FLAG_BAD_LAYOUT);
    return;
  }
  float acc[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) acc[r][c] = 0.f;
  const unsigned int nu = (unsigned int)n;
  for (long long kb = k0; kb < k1; kb += 32 * U) {
    int j[U];
    float a[U][DD];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long k = kb + 32 * u + lane;
      const bool valid = k < k1;
      // a lane past the row's end uses X_0 with zero values
      // clamped into [0, n): whatever the buffer holds, X_j stays in bounds
      j[u] = (int)min(valid ? (unsigned int)__ldg(col + k) : 0u, nu - 1u);
      const T* vk = val + bcsr_val_pos(k, 0, DD);
#pragma unroll
      for (int e = 0; e < DD; ++e) a[u][e] = valid ? bcsr_load(vk + e * 32) : 0.f;
    }
    if constexpr (BcsrX<D>::kCoop) {
      __syncwarp();  // the previous trip has read xs
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < DD; ++q) {
          const int f = q * 32 + lane;
          const int b = f / DD, m = f - b * DD;
          const int jb = __shfl_sync(0xffffffffu, j[u], b);
          xs[u * 32 * DD + f] = __ldg(X + (long long)jb * DD + m);
        }
      __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float x[DD];
      if constexpr (BcsrX<D>::kCoop) {
#pragma unroll
        for (int m = 0; m < DD; ++m) x[m] = xs[u * 32 * DD + lane * DD + m];
      } else if constexpr (DD % 4 == 0) {
        const float4* xp = reinterpret_cast<const float4*>(X + (long long)j[u] * DD);
#pragma unroll
        for (int q = 0; q < DD / 4; ++q) {
          const float4 t = __ldg(xp + q);
          x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
      } else {
        x[0] = __ldg(X + j[u]);  // d = 1
      }
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int c = 0; c < D; ++c) acc[r][c] = fmaf(a[u][r * D + m], x[m * D + c], acc[r][c]);
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
  float* y = Y + i * DD;
  for (int e = lane; e < DD; e += 32) {
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

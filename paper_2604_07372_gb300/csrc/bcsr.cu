// Block-sparse storage for incomplete observations (§4.1: a pair (i, j) is
// observed with probability p; an unobserved pair has A_ij = A_ji = 0).  Only
// observed blocks are stored, so the bytes per A pass are proportional to p.
//
// Layout (NSRGS_BCSR_F32 / NSRGS_BCSR_BF16), block compressed rows of A_off:
// both triangles are kept (A_ji = A_ij^T stored as its own block), so every
// block row is complete and its product Y_i = sum_j A_ij X_j needs no atomics:
// one warp owns row i.  Rows have about the same number of blocks (p(n-1) on
// average), which balances the warps.  Storing both triangles doubles the bytes
// of the observed blocks; it pays against the symmetric panels whenever p < 1/2.
//   [0, 64)          header: int64 n, d, nnzb (number of stored blocks), off_col, off_val
//   [64, ...)        int64 rowptr[n + 1]
//   off_col          int32 col[nnzb], blocks of a row in increasing j
//   off_val          values (float32 or bfloat16) of the nnzb d x d blocks, in
//                    groups of 32 consecutive blocks; within a group element
//                    e = r*d + c of block k sits at e*32 + (k mod 32)
//                    (bcsr_val_pos); the last group is zero-padded to 32 blocks
// A block counts as observed when any of its d*d entries is nonzero.
// Packing reads the strict upper triangle (the canonical list or a dense matrix)
// twice, once to count each row's blocks and once to write them, in column
// order with warp ballots, so the result does not depend on thread timing.
#include <algorithm>

#include "bcsr.cuh"
#include "src.cuh"

namespace nsrgs {

long long bcsr_bytes(int n, int d, int storage, long long nnzb) { return bcsr_bytes_of(n, d, storage, nnzb); }

// Block (min(i, j), max(i, j)) of the strict upper triangle has a nonzero entry.
template <class Src>
__device__ __forceinline__ bool block_observed(const Src& src, int i, int j, int d) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c)
      if (src((long long)a * d + r, (long long)b * d + c) != 0.f) return true;
  return false;
}

// Warp per block row: deg[i] = observed blocks j != i; optionally their total.
template <class Src>
__global__ void __launch_bounds__(256) bcsr_count_kernel(Src src, int n, int d, long long* deg,
                                                          unsigned long long* total) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
    long long cnt = 0;
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      const bool nz = j < n && j != i && block_observed(src, (int)i, j, d);
      cnt += __popc(__ballot_sync(0xffffffffu, nz));
    }
    if (lane == 0) {
      if (deg) deg[i] = cnt;
      if (total) atomicAdd(total, (unsigned long long)cnt);
    }
  }
}

// One CTA: rowptr (at packed + 64) = exclusive scan of deg, written in place over
// deg's copy; header fields filled from the total; the alignment gaps, the
// padding of the last value group and the tail are zeroed (the fill kernel
// then writes the stored blocks), so that a packed buffer is a function of the
// data alone.
__global__ void __launch_bounds__(1024) bcsr_scan_kernel(uint8_t* packed, int n, int d, int storage) {
  long long* rowptr = reinterpret_cast<long long*>(packed + kBcsrHeader);  // holds deg on entry
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const long long per = ((long long)n + blockDim.x - 1) / blockDim.x;
  const long long lo = t * per, hi = std::min<long long>((long long)n, lo + per);
  long long s = 0;
  for (long long i = lo; i < hi; ++i) s += rowptr[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const long long v = part[k];
      part[k] = run;
      run += v;
    }
    long long* hdr = reinterpret_cast<long long*>(packed);
    hdr[0] = n;
    hdr[1] = d;
    hdr[2] = run;
    hdr[3] = bcsr_off_col(n);
    hdr[4] = bcsr_off_val(n, run);
    for (int k = 5; k < kBcsrHeader / 8; ++k) hdr[k] = 0;
  }
  __syncthreads();
  const long long* hdr = reinterpret_cast<const long long*>(packed);
  const long long nnzb = hdr[2];
  long long run = part[t];
  for (long long i = lo; i < hi; ++i) {
    const long long v = rowptr[i];
    rowptr[i] = run;
    run += v;
  }
  if (t == 0) rowptr[n] = nnzb;
  const long long gaps[3][2] = {
      {kBcsrHeader + 8LL * (n + 1), hdr[3]},
      {hdr[3] + 4 * nnzb, hdr[4]},
      {hdr[4] + (nnzb / 32) * 32 * d * d * bcsr_elem_bytes(storage), bcsr_bytes_of(n, d, storage, nnzb)}};
  for (int g = 0; g < 3; ++g)
    for (long long b = gaps[g][0] + t; b < gaps[g][1]; b += blockDim.x) packed[b] = 0;
}

__device__ __forceinline__ void bcsr_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void bcsr_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Warp per block row: writes the row's observed blocks in increasing j.
template <class Src, class T>
__global__ void __launch_bounds__(256) bcsr_fill_kernel(Src src, int n, int d, uint8_t* packed) {
  const long long* hdr = reinterpret_cast<const long long*>(packed);
  const long long* rowptr = reinterpret_cast<const long long*>(packed + kBcsrHeader);
  int* col = reinterpret_cast<int*>(packed + hdr[3]);
  T* val = reinterpret_cast<T*>(packed + hdr[4]);
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
    long long pos = rowptr[i];
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      const bool nz = j < n && j != i && block_observed(src, (int)i, j, d);
      const unsigned int m = __ballot_sync(0xffffffffu, nz);
      if (nz) {
        const long long k = pos + __popc(m & ((1u << lane) - 1u));
        col[k] = j;
        for (int r = 0; r < d; ++r)
          for (int c = 0; c < d; ++c) {
            // A_ij for j > i from the upper triangle; A_ij = (A_ji)^T for j < i
            const float v = j > i ? src(i * (long long)d + r, (long long)j * d + c)
                                  : src((long long)j * d + c, i * (long long)d + r);
            bcsr_store(val + bcsr_val_pos(k, r * d + c, d * d), v);
          }
      }
      pos += __popc(m);
    }
  }
}

// ------------------------------------------------------------------ stream
// Warp per block row (bcsr_row_product), kBcsrWarps warps per CTA.
template <int D, class T>
__global__ void __launch_bounds__(kBcsrWarps * 32) bcsr_stream_kernel(const uint8_t* __restrict__ packed, int n,
                                                                      const float* __restrict__ X,
                                                                      float* __restrict__ Y, const int* skip,
                                                                      Ctl* ctl) {
  __shared__ float xs[kBcsrWarps][BcsrX<D>::kSmemFloats];
  if (*skip) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * kBcsrWarps;
  for (long long i = blockIdx.x * (long long)kBcsrWarps + w; i < n; i += nwarps)
    bcsr_row_product<D, T>(packed, i, X, Y, lane, xs[w], ctl);
}

// ---------------------------------------------------------------- host
bool bcsr_storage(int storage) { return storage == NSRGS_BCSR_F32 || storage == NSRGS_BCSR_BF16; }

static int bcsr_grid(int n) {
  const long long g = ((long long)n + 7) / 8;  // 8 warps per CTA, one row each per sweep
  return (int)std::min<long long>(std::max<long long>(g, 1), 4LL * num_sms());
}
static int bcsr_stream_grid(int n) {
  const long long g = ((long long)n + kBcsrWarps - 1) / kBcsrWarps;
  return (int)std::min<long long>(std::max<long long>(g, 1), 32LL / kBcsrWarps * num_sms());
}

template <class Src>
static cudaError_t bcsr_count_total(Src src, int n, int d, unsigned long long* d_total, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  bcsr_count_kernel<<<bcsr_grid(n), 256, 0, st>>>(src, n, d, nullptr, d_total);
  return cudaGetLastError();
}

template <class Src>
static cudaError_t bcsr_pack(Src src, int n, int d, int storage, uint8_t* packed, cudaStream_t st) {
  long long* deg = reinterpret_cast<long long*>(packed + kBcsrHeader);
  bcsr_count_kernel<<<bcsr_grid(n), 256, 0, st>>>(src, n, d, deg, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bcsr_scan_kernel<<<1, 1024, 0, st>>>(packed, n, d, storage);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (storage == NSRGS_BCSR_BF16)
    bcsr_fill_kernel<Src, __nv_bfloat16><<<bcsr_grid(n), 256, 0, st>>>(src, n, d, packed);
  else
    bcsr_fill_kernel<Src, float><<<bcsr_grid(n), 256, 0, st>>>(src, n, d, packed);
  return cudaGetLastError();
}

cudaError_t bcsr_pack_upper(const float* upper, int n, int d, int storage, void* packed, cudaStream_t st) {
  return bcsr_pack(UpperSrc{upper, n, d}, n, d, storage, reinterpret_cast<uint8_t*>(packed), st);
}
cudaError_t bcsr_pack_dense(const float* A, int n, int d, int storage, void* packed, cudaStream_t st) {
  return bcsr_pack(DenseSrc{A, n, d}, n, d, storage, reinterpret_cast<uint8_t*>(packed), st);
}
cudaError_t bcsr_count_upper(const float* upper, int n, int d, unsigned long long* d_total, cudaStream_t st) {
  return bcsr_count_total(UpperSrc{upper, n, d}, n, d, d_total, st);
}
cudaError_t bcsr_count_dense(const float* A, int n, int d, unsigned long long* d_total, cudaStream_t st) {
  return bcsr_count_total(DenseSrc{A, n, d}, n, d, d_total, st);
}

template <int D>
static cudaError_t bcsr_stream_d(const void* packed, int n, int storage, const float* X, float* Y, const int* skip,
                                 Ctl* ctl, cudaStream_t st) {
  const uint8_t* p = reinterpret_cast<const uint8_t*>(packed);
  if (storage == NSRGS_BCSR_BF16)
    bcsr_stream_kernel<D, __nv_bfloat16><<<bcsr_stream_grid(n), kBcsrWarps * 32, 0, st>>>(p, n, X, Y, skip, ctl);
  else
    bcsr_stream_kernel<D, float><<<bcsr_stream_grid(n), kBcsrWarps * 32, 0, st>>>(p, n, X, Y, skip, ctl);
  return cudaGetLastError();
}

cudaError_t bcsr_stream(const void* packed, int n, int d, int storage, const float* X, float* Y, const int* skip,
                        Ctl* ctl, cudaStream_t st) {
  switch (d) {
    case 1: return bcsr_stream_d<1>(packed, n, storage, X, Y, skip, ctl, st);
    case 2: return bcsr_stream_d<2>(packed, n, storage, X, Y, skip, ctl, st);
    case 3: return bcsr_stream_d<3>(packed, n, storage, X, Y, skip, ctl, st);
    case 4: return bcsr_stream_d<4>(packed, n, storage, X, Y, skip, ctl, st);
    case 5: return bcsr_stream_d<5>(packed, n, storage, X, Y, skip, ctl, st);
    case 6: return bcsr_stream_d<6>(packed, n, storage, X, Y, skip, ctl, st);
    case 7: return bcsr_stream_d<7>(packed, n, storage, X, Y, skip, ctl, st);
    case 8: return bcsr_stream_d<8>(packed, n, storage, X, Y, skip, ctl, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nsrgs

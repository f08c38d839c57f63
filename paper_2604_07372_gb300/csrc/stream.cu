// Single-instance launch of the symmetric read-once A-stream Y = A_off X
// (the kernel body is in panel.cuh), and the dense plain form.
#include "panel.cuh"

namespace nsrgs {

struct StreamArgs {
  const uint8_t* packed;
  const float* X;  // padded, xpad_rows(n, D) x D
  float* Y;        // padded accumulator, zero on entry
  Ctl* ctl;
  const int* skip;  // the launch does nothing when *skip != 0 (set by earlier launches)
  PanelGeom g;
};

// One instance taken from the kernel parameters.
struct SingleSrc {
  const StreamArgs* a;
  __device__ __forceinline__ int count() const { return 1; }
  __device__ __forceinline__ int find(long long) const { return 0; }
  __device__ __forceinline__ long long base(int i) const { return i == 0 ? 0 : a->g.total_steps; }
  __device__ __forceinline__ InstView view(int) const {
    InstView v;
    v.packed = a->packed;
    v.X = a->X;
    v.Y = a->Y;
    v.ctl = a->ctl;
    v.g = a->g;
    v.skip = false;
    return v;
  }
};

template <int D, int ST>
__global__ void __launch_bounds__(PCfg<D, ST>::THREADS, 1) panel_stream_kernel(const __grid_constant__ StreamArgs a) {
  if (*a.skip) return;  // written only by earlier launches: uniform
  SingleSrc src{&a};
  panel_stream_body<D, ST>(src, a.g.total_steps);
}

// ------------------------------------------------------------ dense form
// Y = A_off X with A_off the full nd x nd matrix (diagonal blocks zero), no
// symmetric reuse: the plain form the symmetric layouts are compared with, and
// the path for block sizes the symmetric layouts do not cover.  CTA = 64 rows;
// thread (row, quarter) sums over every 4th float4 of its row.
template <int DMAX>
__global__ void __launch_bounds__(256) dense_stream_kernel(const float* __restrict__ A, int N, int pitch, int D,
                                                           const float* __restrict__ X, float* __restrict__ Y,
                                                           const int* skip) {
  if (*skip) return;
  __shared__ __align__(16) float xs[64 * DMAX];
  const int r = blockIdx.x * 64 + (threadIdx.x >> 2);
  const int qtr = threadIdx.x & 3;
  float acc[DMAX];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) acc[k] = 0.f;
  for (int c0 = 0; c0 < N; c0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * D; e += 256) {
      const int c = c0 + e / D;
      xs[e] = (c < N) ? X[(long long)c0 * D + e] : 0.f;
    }
    __syncthreads();
    if (r < N) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int cl = s * 16 + qtr * 4;
        const int c = c0 + cl;
        if (c < pitch) {
          const float4 v = *reinterpret_cast<const float4*>(A + (long long)r * pitch + c);
          const float av[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < DMAX; ++k)
              if (k < D) acc[k] = fmaf(av[u], xs[(cl + u) * D + k], acc[k]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 1);
    acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 2);
  }
  if (r < N && qtr == 0)
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
      if (k < D) Y[(long long)r * D + k] = acc[k];
}

// ------------------------------------------------------------- launchers
// Opt-in to the kernel's dynamic shared memory; called outside of any stream
// capture (cudaFuncSetAttribute is a device-wide setting, idempotent).
template <int D, int ST>
static cudaError_t prepare_panel() {
  using C = PCfg<D, ST>;
  return cudaFuncSetAttribute(panel_stream_kernel<D, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
}

template <int D, int ST>
static cudaError_t launch_panel(const StreamArgs& a, cudaStream_t st) {
  using C = PCfg<D, ST>;
  if (a.g.n < 0) return prepare_panel<D, ST>();  // preparation request
  panel_stream_kernel<D, ST><<<num_sms(), C::THREADS, C::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_panel_st(const StreamArgs& a, cudaStream_t st) {
  switch (a.g.storage) {
    case NSRGS_F32: return launch_panel<D, NSRGS_F32>(a, st);
    case NSRGS_BF16: return launch_panel<D, NSRGS_BF16>(a, st);
    case NSRGS_FP8E4M3:
      if constexpr (D <= 4) return launch_panel<D, NSRGS_FP8E4M3>(a, st);
      break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t stream_panel(const void* packed, const PanelGeom& g, const float* X, float* Y, Ctl* ctl,
                         const int* skip, cudaStream_t st) {
  StreamArgs a{reinterpret_cast<const uint8_t*>(packed), X, Y, ctl, skip, g};
  switch (g.D) {
    case 1: return launch_panel_st<1>(a, st);
    case 2: return launch_panel_st<2>(a, st);
    case 3: return launch_panel_st<3>(a, st);
    case 4: return launch_panel_st<4>(a, st);
    case 5: return launch_panel_st<5>(a, st);
    case 6: return launch_panel_st<6>(a, st);
    case 7: return launch_panel_st<7>(a, st);
    case 8: return launch_panel_st<8>(a, st);
  }
  return cudaErrorInvalidValue;
}

// Sets the launch attributes of the stream kernel for this geometry.
cudaError_t stream_panel_prepare(const PanelGeom& g) {
  PanelGeom h = g;
  h.n = -1;
  return stream_panel(nullptr, h, nullptr, nullptr, nullptr, nullptr, 0);
}

long long dense_pitch(int n, int d);

// Y = A_off X for an X with `width` columns (d for the method, p for the Stiefel form).
cudaError_t stream_dense_width(const void* packed, int n, int d, int width, const float* X, float* Y,
                               const int* skip, cudaStream_t st) {
  const int N = n * d;
  const int pitch = (int)dense_pitch(n, d);
  dim3 grid((N + 63) / 64);
  const float* A = reinterpret_cast<const float*>(packed);
  const int w = width;
  if (w <= 4) dense_stream_kernel<4><<<grid, 256, 0, st>>>(A, N, pitch, w, X, Y, skip);
  else if (w <= 8) dense_stream_kernel<8><<<grid, 256, 0, st>>>(A, N, pitch, w, X, Y, skip);
  else if (w <= 16) dense_stream_kernel<16><<<grid, 256, 0, st>>>(A, N, pitch, w, X, Y, skip);
  else if (w <= 32) dense_stream_kernel<32><<<grid, 256, 0, st>>>(A, N, pitch, w, X, Y, skip);
  else dense_stream_kernel<64><<<grid, 256, 0, st>>>(A, N, pitch, w, X, Y, skip);
  return cudaGetLastError();
}

cudaError_t stream_dense(const void* packed, int n, int d, const float* X, float* Y, const int* skip,
                         cudaStream_t st) {
  return stream_dense_width(packed, n, d, d, X, Y, skip, st);
}

}  // namespace nsrgs

// Single-instance launch of the symmetric read-once A-stream Y = A_off X
// (the kernel body is in panel.cuh), and the dense plain form.
#include "blockops.cuh"
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
  static constexpr bool kStreamOnce = true;  // A is read once per pass: L2 evict-first
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

// ------------------------------------------------------ fused iteration loop
// All T iterations of Algorithm 2 on the panel layout in ONE launch: per
// iteration the A stream Y = A_off X^t (the tuned pipeline, whose stage and ring
// positions carry over from pass to pass), a grid-wide barrier, each CTA's share
// of the block updates (gradient, tangent projection, step, K Newton-Schulz
// steps; Y cleared), and a second barrier whose last arrival finishes the update
// norm and the stop test before the next pass.  No kernel boundary, launch gap or
// pipeline set-up remains between iterations.  The grid is one CTA per SM (the
// stream's shared memory admits one), all resident at once; every barrier wait
// is bounded (a timeout sets FLAG_TIMEOUT and the CTA leaves).
struct LoopArgs {
  StreamArgs s;     // packed A, Y (zero on entry and on exit), ctl, skip; s.X unused
  float* X0;        // X^t for even t
  float* X1;        // X^t for odd t
  float eta;
  int K;
  int safeguard;
  int T;
  double tol;       // > 0: stop after the first iteration whose update norm is below it
};


// Grid-wide barrier on a monotonic arrival counter of the control block: barrier
// number k of a launch completes when the counter reaches (k + 1) * gridDim.x
// (the counter starts at zero with the call's control-block reset and is never
// wound back, so no CTA has to reset anything).  Arrival is a release add, the
// wait an acquire poll, bounded; returns false (in every thread of the CTA)
// after a timeout.  Every thread calls it.
__device__ __forceinline__ bool grid_barrier_bounded(Ctl* ctl, unsigned int target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();  // the CTA's global writes and reductions before the arrival
    unsigned int* cnt = &ctl->gbar_count;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt) : "memory");
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
    if ((int)(v - target) < 0) {
      const uint64_t t0 = globaltimer_ns();
      while (true) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
        if ((int)(v - target) >= 0) break;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          ok = 0;
          atomicOr(&ctl->flags, FLAG_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();  // later reads of the CTA see the other CTAs' writes (no stale L1 lines)
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Generic-proxy writes of X by this thread become visible to the TMA engine
// (the async proxy) that reads X rows in the next pass.
__device__ __forceinline__ void fence_x_for_tma() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

template <int D, int ST>
__global__ void __launch_bounds__(PCfg<D, ST>::THREADS, 1) panel_loop_kernel(const __grid_constant__ LoopArgs a) {
  Ctl* ctl = a.s.ctl;
  // uniform: both are written only by earlier launches
  if (*a.s.skip || (*reinterpret_cast<volatile unsigned int*>(&ctl->flags) & FLAG_TIMEOUT)) return;
  __shared__ double sh[32];
  __shared__ int s_stop;
  const long long total = a.s.g.total_steps;
  const long long g0 = total * blockIdx.x / gridDim.x;
  const long long g1 = total * (blockIdx.x + 1) / gridDim.x;
  const int n = a.s.g.n;
  const long long b0 = (long long)n * blockIdx.x / gridDim.x;
  const long long b1 = (long long)n * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) panel_init_barriers<D, ST>();
  __syncthreads();
  PanelPipe pp;
  StreamArgs sa = a.s;
  for (int t = 0; t < a.T; ++t) {
    const float* Xt = (t & 1) ? a.X1 : a.X0;
    float* Xn = (t & 1) ? a.X0 : a.X1;
    if (g0 < g1) {
      sa.X = Xt;
      SingleSrc src{&sa};
      panel_stream_range<D, ST>(src, g0, g1, pp, RES_RING);
    }
    if (!grid_barrier_bounded(ctl, (2u * t + 1u) * gridDim.x)) return;
    // this CTA's blocks of Algorithm 2's update
    double diff2 = 0.0;
    unsigned int flags = 0;
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x)
      block_update<D>(Xt, a.s.Y, Xn, i, n, a.eta, a.K, a.safeguard != 0, diff2, flags);
    if (flags) atomicOr(&ctl->flags, flags);
    fence_x_for_tma();
    // update-norm partials into the accumulator of this iteration's parity; the
    // other one is cleared for the next iteration (nobody adds to it before the
    // next first barrier, which orders the clearing)
    const double bs = block_sum(diff2, sh);
    if (threadIdx.x == 0) {
      atomicAdd(&ctl->upd_acc2[t & 1], bs);
      if (blockIdx.x == 0) ctl->upd_acc2[(t + 1) & 1] = 0.0;
    }
    if (!grid_barrier_bounded(ctl, (2u * t + 2u) * gridDim.x)) return;
    // every CTA reads the complete sum and takes the same stop decision
    if (threadIdx.x == 0) {
      const double tot = *reinterpret_cast<volatile double*>(&ctl->upd_acc2[t & 1]);
      const double un = sqrt(tot / ((double)n * D));
      const int stop = (a.tol > 0.0 && un < a.tol) ? 1 : 0;
      if (blockIdx.x == 0) {
        ctl->last_upd = un;
        ctl->iters_done += 1;
        if (stop) ctl->stop = 1;
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
  }
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
  cudaError_t e = cudaFuncSetAttribute(panel_stream_kernel<D, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  if constexpr (D <= 7)
    return cudaFuncSetAttribute(panel_loop_kernel<D, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  return cudaSuccess;
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

template <int D, int ST>
static cudaError_t launch_loop(const LoopArgs& a, cudaStream_t st) {
  using C = PCfg<D, ST>;
  panel_loop_kernel<D, ST><<<num_sms(), C::THREADS, C::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_loop_st(const LoopArgs& a, cudaStream_t st) {
  switch (a.s.g.storage) {
    case NSRGS_F32: return launch_loop<D, NSRGS_F32>(a, st);
    case NSRGS_BF16: return launch_loop<D, NSRGS_BF16>(a, st);
    case NSRGS_FP8E4M3:
      if constexpr (D <= 4) return launch_loop<D, NSRGS_FP8E4M3>(a, st);
      break;
  }
  return cudaErrorInvalidValue;
}

// T iterations on the panel layout in one launch, from X0 (X^t alternates between
// X0 and X1; ctl->iters_done counts the iterations run).
cudaError_t iterate_panel_loop(const void* packed, const PanelGeom& g, float* X0, float* X1, float* Y, float eta, int K,
                               int safeguard, int T, double tol, Ctl* ctl, const int* skip, cudaStream_t st) {
  LoopArgs a{StreamArgs{reinterpret_cast<const uint8_t*>(packed), X0, Y, ctl, skip, g}, X0, X1, eta, K, safeguard, T,
             tol};
  switch (g.D) {
    case 1: return launch_loop_st<1>(a, st);
    case 2: return launch_loop_st<2>(a, st);
    case 3: return launch_loop_st<3>(a, st);
    case 4: return launch_loop_st<4>(a, st);
    case 5: return launch_loop_st<5>(a, st);
    case 6: return launch_loop_st<6>(a, st);
    case 7: return launch_loop_st<7>(a, st);
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

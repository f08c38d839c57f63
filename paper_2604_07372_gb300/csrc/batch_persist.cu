// Persistent batched form: ONE launch runs every instance's whole solve --
// spectral start (subspace passes, the algebraic top-d test, the exact
// blockwise sign) and T iterations of Algorithm 2 -- with no grid-wide step.
//
// The grid is one CTA per SM.  A CTA takes instances from a device work counter
// in the host's order (largest first, so the long solves start at once and the
// short ones fill the tail) and runs each instance alone: per A pass it streams
// the instance's panels through the same tuned pipeline as the single-instance
// kernel (panel_stream_range: TMA producer, consumer warps, reducer warp), and
// between passes its threads do the d x d work of the pass (Gram, Cholesky,
// basis update and residual; or the per-block update and the update norm) with
// CTA-local reductions.  An instance therefore needs no barrier beyond the
// CTA's own __syncthreads, and the pipeline's barriers are set up once per CTA:
// its stage and ring positions carry over from pass to pass and instance to
// instance.
//
// Residency: an instance whose panels, stored densely step after step with
// their X rows, fit in the CTA's stage space is loaded into shared memory on
// its first A pass and read from there on every later pass (only the X rows of
// each step are copied again), so a small instance touches HBM for its A once
// per solve instead of once per pass.
#include <math.h>

#include "batch.cuh"
#include "blockops.cuh"
#include "panel.cuh"

namespace nsrgs {

// One instance as the panel source of a CTA-local pass.
struct OneSrc {
  InstView v;
  long long steps;
  __device__ __forceinline__ int count() const { return 1; }
  __device__ __forceinline__ int find(long long) const { return 0; }
  __device__ __forceinline__ long long base(int i) const { return i == 0 ? 0 : steps; }
  __device__ __forceinline__ InstView view(int) const { return v; }
};

struct PersistArgs {
  const BatchDesc* descs;
  const int* order;  // instance indices in the order CTAs take them
  int count;
  int* next;         // work counter, zero at launch
};

// CTA-wide sums of NV doubles held by every thread; the totals land in out[]
// (shared) and are valid in every thread on return.
template <int NV>
__device__ __forceinline__ void cta_sums(double (&v)[NV], double* red, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w * NV + k] = v[k];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double s = 0.0;
    for (int ww = 0; ww < nw; ++ww) s += red[ww * NV + k];
    out[k] = s;
  }
  __syncthreads();
}

// Generic-proxy writes of X by this thread become visible to the TMA engine
// (the async proxy) that reads X rows in the next A pass.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Shared scratch of one CTA: per-warp partials and the pass's d x d results.
template <int D>
struct PersistShared {
  static constexpr int DD = D * D;
  double red[32 * 2 * DD];  // up to 32 warps x 2 D^2 partials
  double tot[2 * DD];       // CTA totals
  double rinv[DD];          // chol(W^T W)^{-1}
  double H[DD];             // V^T W
  double tmp[DD];           // Cholesky / bisection scratch
  double h2;                // ||H||_F^2
  double new_shift;         // the larger shift of a restart
  unsigned int flags;       // FLAG_* bits of the running pass
  int decision;             // thread 0's verdict after a spectral pass
  int k;                    // work item taken by thread 0
};

enum : int { SPEC_GO_ON = 0, SPEC_DONE = 1, SPEC_RESTART = 2 };

template <int D, int ST>
__device__ bool persist_instance(const BatchDesc& dsc, PanelPipe& pp, PersistShared<D>& sh) {
  constexpr int DD = D * D;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = dsc.g.n;
  const long long rows = (long long)n * D;
  const long long vec = (long long)xpad_rows(n, D) * D;
  Ctl* c = dsc.ctl;
  float* X[2] = {dsc.X[0], dsc.X[1]};
  float* Y = dsc.Y;
  float* W = dsc.W;

  // ------------------------------------------------------------- admit
  for (long long e = tid; e < vec; e += nt) {
    Y[e] = 0.f;
    if (e >= rows * D) {
      X[0][e] = 0.f;
      X[1][e] = 0.f;
    } else {
      X[0][e] = dsc.start_given ? dsc.Xout[e] : spec_v0_entry(e);
    }
  }
  if (tid == 0) {
    sh.flags = 0u;
    c->upd_acc = 0.0;
    c->last_upd = 0.0;
    c->spec_res = 0.0;
    c->counter = 0u;
    c->iters_done = 0;
    c->stop = 0;
    c->flags = 0u;
    c->spec_iters = 0;
    c->spec_stop = 0;
    c->spec_skip = 0;
    c->spec_restart = 0;
    c->spec_round = 0;
    c->spec_prev = 0;
    c->phase = dsc.start_given ? PHASE_ITER : PHASE_SPEC;
  }
  __syncthreads();

  bool loaded = false;
  bool failed = false;
  // One A pass: Y = A_off X (Y is zero on entry).
  auto a_pass = [&](const float* Xv) {
    fence_proxy_async_global();
    __syncthreads();
    OneSrc src;
    src.v.packed = dsc.packed;
    src.v.X = Xv;
    src.v.Y = Y;
    src.v.ctl = c;
    src.v.g = dsc.g;
    src.v.skip = false;
    src.steps = dsc.g.total_steps;
    const int mode = dsc.resident ? (loaded ? RES_KEEP : RES_LOAD) : RES_RING;
    panel_stream_range<D, ST>(src, 0, dsc.g.total_steps, pp, mode);
    loaded = true;
    __syncthreads();
    failed = (*reinterpret_cast<volatile unsigned int*>(&c->flags) & (FLAG_TIMEOUT | FLAG_BAD_LAYOUT)) != 0u;
    __syncthreads();
  };
  // Gram of W = Y + c V (ortho: W = V, no product) -> R^{-1}, H (shared); Y cleared.
  auto gram = [&](const float* V, bool ortho, float shift) {
    double acc[2 * DD];
#pragma unroll
    for (int o = 0; o < 2 * DD; ++o) acc[o] = 0.0;
    for (long long r = tid; r < rows; r += nt) {
      float v[D], w[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[k] = V[r * D + k];
        w[k] = ortho ? v[k] : Y[r * D + k] + shift * v[k];
        W[r * D + k] = w[k];
        Y[r * D + k] = 0.f;
      }
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          acc[a * D + b] += (double)w[a] * (double)w[b];
          acc[DD + a * D + b] += (double)v[a] * (double)w[b];
        }
    }
    cta_sums<2 * DD>(acc, sh.red, sh.tot);
    if (tid == 0) {
      chol_inv(sh.tot, sh.rinv, D, sh.tmp);
      double h2 = 0.0;
      for (int o = 0; o < DD; ++o) {
        sh.H[o] = sh.tot[DD + o];
        h2 += sh.H[o] * sh.H[o];
      }
      sh.h2 = h2;
    }
    __syncthreads();
  };
  // V_new = W R^{-1}; returns the residual ||W - V H||_F^2 (every thread).
  auto update = [&](const float* V, float* Vn) -> double {
    double res[1] = {0.0};
    for (long long r = tid; r < rows; r += nt) {
      double v[D], w[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[k] = V[r * D + k];
        w[k] = W[r * D + k];
      }
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        double nv = 0.0, vh = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          nv += w[k] * sh.rinv[k * D + cc];
          vh += v[k] * sh.H[k * D + cc];
        }
        Vn[r * D + cc] = (float)nv;
        const double e = w[cc] - vh;
        res[0] += e * e;
      }
    }
    cta_sums<1>(res, sh.red, sh.tot);
    return sh.tot[0];
  };

  // ------------------------------------------------- spectral start
  int spec_total = 0, s = 0;
  if (!dsc.start_given) {
    float shift = 1.f;  // W = A_off V + V: subspace iteration on A itself
    int round = 0;
    gram(X[0], true, 1.f);
    update(X[0], X[1]);
    for (;;) {
      if (spec_total >= dsc.smax) break;
      const float* V = X[(s + 1) & 1];
      float* Vn = X[s & 1];
      a_pass(V);
      if (failed) return false;
      gram(V, false, shift);
      const double tot = update(V, Vn);
      ++s;
      ++spec_total;
      if (tid == 0) {
        const double rel = sqrt(tot / fmax(sh.h2, 1e-300));
        c->spec_res = rel;
        sh.decision = SPEC_GO_ON;
        if (rel <= dsc.spec_tol) {
          const double c2 = spec_shift_after(sh.H, D, (double)shift, sh.tmp);
          if (c2 == 0.0) {
            c->spec_stop = 1;
            sh.decision = SPEC_DONE;
          } else if (round >= kSpecMaxRestarts || spec_total >= dsc.smax) {
            sh.decision = SPEC_DONE;  // spec_stop stays clear: reported as not converged
          } else {
            sh.new_shift = c2;
            sh.flags |= FLAG_SPEC_SHIFTED;
            sh.decision = SPEC_RESTART;
          }
        }
      }
      __syncthreads();
      const int dec = sh.decision;
      if (dec == SPEC_DONE) break;
      if (dec == SPEC_RESTART) {
        // the start again, orthonormalised under the larger shift
        shift = (float)sh.new_shift;
        ++round;
        __syncthreads();
        for (long long e = tid; e < rows * D; e += nt) X[0][e] = spec_v0_entry(e);
        __syncthreads();
        gram(X[0], true, 1.f);
        update(X[0], X[1]);
        s = 0;
      }
    }
    // X^0_i = sgn(V_i), exact float64 polar per block (Algorithm 2's start)
    const float* Vf = s > 0 ? X[(s - 1) & 1] : X[1];
    for (int i = tid; i < n; i += nt) {
      double M[D][D], Q[D][D];
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int cc = 0; cc < D; ++cc) M[r][cc] = Vf[((long long)i * D + r) * D + cc];
      polar_fp64<D>(M, Q);
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
          X[0][((long long)i * D + r) * D + cc] = (float)Q[r][cc];
          if (dsc.T == 0) dsc.Xout[((long long)i * D + r) * D + cc] = (float)Q[r][cc];
        }
    }
    __syncthreads();
  }

  // ----------------------------------------------------- iterations
  int it = 0;
  double un = 0.0;
  for (; it < dsc.T;) {
    const float* Xt = X[it & 1];
    float* Xn = X[(it + 1) & 1];
    a_pass(Xt);
    if (failed) return false;
    double part[1] = {0.0};
    unsigned int fl = 0u;
    for (int i = tid; i < n; i += nt) block_update<D>(Xt, Y, Xn, i, n, dsc.eta, dsc.K, dsc.safeguard != 0, part[0], fl);
    if (fl) atomicOr(&sh.flags, fl);
    cta_sums<1>(part, sh.red, sh.tot);
    un = sqrt(sh.tot[0] / ((double)n * D));
    ++it;
    if ((dsc.tol > 0.0 && un < dsc.tol) || (sh.flags & FLAG_NONFINITE)) break;
  }
  if (dsc.T > 0 || dsc.start_given) {
    const float* Xf = X[it & 1];
    for (long long e = tid; e < rows * D; e += nt) dsc.Xout[e] = Xf[e];
  }
  if (tid == 0) {
    c->iters_done = it;
    c->last_upd = un;
    c->stop = (dsc.tol > 0.0 && un < dsc.tol && it > 0) ? 1 : 0;
    c->spec_iters = s;
    c->spec_prev = spec_total - s;
    c->flags |= sh.flags;
    c->phase = PHASE_DONE;
  }
  __syncthreads();
  return true;
}

template <int D, int ST>
__global__ void __launch_bounds__(PCfg<D, ST>::THREADS, 1) batch_persist_kernel(const __grid_constant__ PersistArgs a) {
  __shared__ PersistShared<D> sh;
  if (threadIdx.x == 0) panel_init_barriers<D, ST>();
  __syncthreads();
  PanelPipe pp;
  for (;;) {
    if (threadIdx.x == 0) sh.k = atomicAdd(a.next, 1);
    __syncthreads();
    const int k = sh.k;
    __syncthreads();
    if (k >= a.count) break;
    // a pass that timed out or found a bad layout leaves this CTA's pipeline in an
    // unknown state: the CTA stops taking work (the host reports the flag)
    if (!persist_instance<D, ST>(a.descs[a.order[k]], pp, sh)) break;
  }
}

// ---------------------------------------------------------------- host
// Bytes of an instance's panels stored densely step after step with the X rows
// of each step (the resident layout), and whether they fit a CTA's stage space.
template <int D, int ST>
static bool fits_resident_t(const PanelGeom& g) {
  using C = PCfg<D, ST>;
  const long long dense = g.panel_bytes + g.total_steps * (long long)C::STAGE_X;
  return dense <= (long long)C::OFF_RING;
}

template <int D, int ST>
static cudaError_t launch_persist_t(const PersistArgs& a, cudaStream_t st, bool prepare) {
  using C = PCfg<D, ST>;
  static_assert(C::SMEM + sizeof(PersistShared<D>) <= 227 * 1024, "shared memory");
  if (prepare)
    return cudaFuncSetAttribute(batch_persist_kernel<D, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  batch_persist_kernel<D, ST><<<num_sms(), C::THREADS, C::SMEM, st>>>(a);
  return cudaGetLastError();
}

#define NSRGS_PERSIST_DISPATCH(d, storage, F)                                   \
  switch (d * 8 + storage) {                                                    \
    case 1 * 8 + NSRGS_F32: return F(1, NSRGS_F32);                             \
    case 1 * 8 + NSRGS_BF16: return F(1, NSRGS_BF16);                           \
    case 1 * 8 + NSRGS_FP8E4M3: return F(1, NSRGS_FP8E4M3);                     \
    case 2 * 8 + NSRGS_F32: return F(2, NSRGS_F32);                             \
    case 2 * 8 + NSRGS_BF16: return F(2, NSRGS_BF16);                           \
    case 2 * 8 + NSRGS_FP8E4M3: return F(2, NSRGS_FP8E4M3);                     \
    case 3 * 8 + NSRGS_F32: return F(3, NSRGS_F32);                             \
    case 3 * 8 + NSRGS_BF16: return F(3, NSRGS_BF16);                           \
    case 3 * 8 + NSRGS_FP8E4M3: return F(3, NSRGS_FP8E4M3);                     \
    case 4 * 8 + NSRGS_F32: return F(4, NSRGS_F32);                             \
    case 4 * 8 + NSRGS_BF16: return F(4, NSRGS_BF16);                           \
    case 4 * 8 + NSRGS_FP8E4M3: return F(4, NSRGS_FP8E4M3);                     \
  }

bool persist_fits_resident(const PanelGeom& g) {
#define F(DD, SS) fits_resident_t<DD, SS>(g)
  NSRGS_PERSIST_DISPATCH(g.D, g.storage, F)
#undef F
  return false;
}

cudaError_t batch_persist(const BatchDesc* descs, const int* order, int count, int* next, int d, int storage,
                          cudaStream_t st, bool prepare) {
  PersistArgs a{descs, order, count, next};
#define F(DD, SS) launch_persist_t<DD, SS>(a, st, prepare)
  NSRGS_PERSIST_DISPATCH(d, storage, F)
#undef F
  return cudaErrorInvalidValue;
}

}  // namespace nsrgs

// Per-block and reduction kernels around the A stream:
//  * the iteration epilogue of Algorithm 2 (gradient, tangent projection, step,
//    K Newton-Schulz steps, update norm, status flags);
//  * the spectral initialisation's subspace-iteration steps (float64 Gram,
//    Cholesky, V <- W R^{-1}, residual) and the exact blockwise matrix sign;
//  * the distance d_F(X, Y) of §1.4.
#include <math.h>

#include "blockops.cuh"

namespace nsrgs {

constexpr int kDmaxSmall = 8;  // thread-per-block kernels are instantiated for d <= 8

// ------------------------------------------------------ iteration epilogue
// Thread i handles block i (block_update: Algorithm 2's loop body); the last
// CTA finishes the update norm ||X^{t+1} - X^t||_F / sqrt(nd) and the stop test.
template <int D>
__global__ void __launch_bounds__(128) epilogue_kernel(const float* __restrict__ X, float* __restrict__ Y,
                                                       float* __restrict__ Xout, int n, float eta, int K,
                                                       int safeguard, double tol, Ctl* ctl, double* upd_out) {
  __shared__ double sh[32];
  if (ctl->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double diff2 = 0.0;
  unsigned int flags = 0;
  if (i < n) block_update<D>(X, Y, Xout, i, n, eta, K, safeguard != 0, diff2, flags);
  if (flags) atomicOr(&ctl->flags, flags);
  const double bs = block_sum(diff2, sh);
  if (threadIdx.x == 0) atomicAdd(&ctl->upd_acc, bs);
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) {
      const double tot = atomicAdd(&ctl->upd_acc, 0.0);
      const double un = sqrt(tot / ((double)n * D));
      ctl->last_upd = un;
      ctl->iters_done += 1;
      if (tol > 0.0 && un < tol) ctl->stop = 1;
      ctl->upd_acc = 0.0;
      ctl->counter = 0u;
      if (upd_out) *upd_out = un;
    }
  }
}

// ------------------------------------------------ GPM (comparison method)
// Generalised power method step, the paper's comparison method (read as
// X_i <- sgn(sum_j A_ij X_j) with A_ii = I): M = Y_i + X_i, then the exact
// per-block sign by a float32 one-sided Jacobi SVD (a batched per-block SVD,
// the cost NS-RGS removes).  Same update-norm / stop bookkeeping as the epilogue.
template <int D>
__global__ void __launch_bounds__(128) gpm_epilogue_kernel(const float* __restrict__ X, float* __restrict__ Y,
                                                           float* __restrict__ Xout, int n, double tol, Ctl* ctl) {
  __shared__ double sh[32];
  if (ctl->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double diff2 = 0.0;
  unsigned int flags = 0;
  if (i < n) {
    float M[D][D], x[D][D], Q[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const long long e = ((long long)i * D + r) * D + c;
        x[r][c] = X[e];
        M[r][c] = Y[e] + x[r][c];
        Y[e] = 0.f;
      }
    polar_fp32<D>(M, Q);
    bool finite = true;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        finite = finite && isfinite(Q[r][c]);
        Xout[((long long)i * D + r) * D + c] = Q[r][c];
        const double dd = (double)Q[r][c] - (double)x[r][c];
        diff2 += dd * dd;
      }
    if (!finite) flags |= FLAG_NONFINITE;
  }
  if (flags) atomicOr(&ctl->flags, flags);
  const double bs = block_sum(diff2, sh);
  if (threadIdx.x == 0) atomicAdd(&ctl->upd_acc, bs);
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) {
      const double tot = atomicAdd(&ctl->upd_acc, 0.0);
      const double un = sqrt(tot / ((double)n * D));
      ctl->last_upd = un;
      ctl->iters_done += 1;
      if (tol > 0.0 && un < tol) ctl->stop = 1;
      ctl->upd_acc = 0.0;
      ctl->counter = 0u;
    }
  }
}

// ------------------------------------------- spectral init: subspace steps
// Deterministic start V0 (any full-rank start works; entries uniform in (-1, 1)).
// With shift_slot non-null the spectral shift starts at c = 1 (W = A_off V + V,
// i.e. subspace iteration on A itself, A_ii = I).
__global__ void spec_v0_kernel(float* V, long long rows, int D, double* shift_slot) {
  const long long total = rows * D;
  if (shift_slot && blockIdx.x == 0 && threadIdx.x == 0) *shift_slot = 1.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    V[e] = spec_v0_entry(e);
}

// W = Y + c V (written to W, Y zeroed), partial sums of W^T W and V^T W;
// the last CTA reduces them, forms H = V^T W, ||H||_F^2 and Rinv = chol(W^T W)^{-1}.
// c is `shift` for the orthonormalising pass (dev_shift = 0) and the current
// shift s.scal[3] otherwise.  A pass after a failed algebraic top-d test
// (ctl->spec_restart) takes W = V^0 instead: the start again, to be
// orthonormalised under the new shift.
template <int D>
__global__ void __launch_bounds__(256) spec_gram_kernel(const float* __restrict__ V, float* __restrict__ Y,
                                                        float* __restrict__ W, long long rows, float shift,
                                                        int dev_shift, SpecScratch s, Ctl* ctl) {
  __shared__ double sh[32];
  if (ctl->spec_skip) return;
  const bool restart = dev_shift && ctl->spec_restart;
  const float c = dev_shift ? (float)s.scal[3] : shift;
  double ww[D][D], vw[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) ww[a][b] = vw[a][b] = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    float v[D], w[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = V[r * D + k];
      w[k] = restart ? spec_v0_entry(r * D + k) : Y[r * D + k] + c * v[k];
      W[r * D + k] = w[k];
      Y[r * D + k] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        ww[a][b] += (double)w[a] * (double)w[b];
        vw[a][b] += (double)v[a] * (double)w[b];
      }
  }
  double* part = s.partials + (long long)blockIdx.x * 2 * D * D;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const double x1 = block_sum(ww[a][b], sh);
      const double x2 = block_sum(vw[a][b], sh);
      if (threadIdx.x == 0) {
        part[a * D + b] = x1;
        part[D * D + a * D + b] = x2;
      }
    }
  if (last_block(&ctl->counter)) {
    for (int o = threadIdx.x; o < 2 * D * D; o += blockDim.x) {
      double acc = 0.0;
      for (unsigned int bb = 0; bb < gridDim.x; ++bb) acc += s.partials[(long long)bb * 2 * D * D + o];
      if (o < D * D) s.WW[o] = acc; else s.H[o - D * D] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double h2 = 0.0;
      for (int o = 0; o < D * D; ++o) h2 += s.H[o] * s.H[o];
      s.scal[0] = h2;
      chol_inv(s.WW, s.Rinv, D, s.M);
      s.scal[2] = 0.0;
      ctl->counter = 0u;
    }
  }
}

// Vnew = W Rinv and the residual ||W - V H||_F; the last CTA finishes the
// residual ||A V - V H||_F / ||H||_F and, when it is <= tol, applies the
// algebraic top-d test (spec_finish_pass).
template <int D>
__global__ void __launch_bounds__(256) spec_update_kernel(const float* __restrict__ V, const float* __restrict__ W,
                                                          float* __restrict__ Vnew, long long rows, SpecScratch s,
                                                          double tol, int count_pass, Ctl* ctl) {
  __shared__ double sh[32];
  __shared__ double rinv[D * D], hh[D * D];
  if (ctl->spec_skip) return;
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) {
    rinv[o] = s.Rinv[o];
    hh[o] = s.H[o];
  }
  __syncthreads();
  double res = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    double v[D], w[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = V[r * D + k];
      w[k] = W[r * D + k];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double nv = 0.0, vh = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        nv += w[k] * rinv[k * D + c];
        vh += v[k] * hh[k * D + c];
      }
      Vnew[r * D + c] = (float)nv;
      const double e = w[c] - vh;
      res += e * e;
    }
  }
  const double bs = block_sum(res, sh);
  if (threadIdx.x == 0) atomicAdd(&s.scal[2], bs);
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) {
      const double tot = atomicAdd(&s.scal[2], 0.0);
      ctl->counter = 0u;
      if (count_pass) spec_finish_pass(tot, D, tol, s, ctl, spec_floor_max(count_pass));
    }
  }
}

// X0_i = sgn(V_i): exact float64 polar of each block (Algorithm 2's X^0).
template <int D>
__global__ void polar_blocks_kernel(const float* __restrict__ V, float* __restrict__ X0, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double M[D][D], Q[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) M[r][c] = V[((long long)i * D + r) * D + c];
  polar_fp64<D>(M, Q);
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) X0[((long long)i * D + r) * D + c] = (float)Q[r][c];
}

// ------------------------------------------------------------- d_F(X, Y)
// M = Y^T X (float64); the last CTA forms Q = sgn(M) (the minimiser of
// ||X - Y Q||_F over O(d), proof of Lemma 7.4).
template <int D>
__global__ void __launch_bounds__(256) cross_gram_kernel(const float* __restrict__ X, const float* __restrict__ Yv,
                                                         long long rows, SpecScratch s, Ctl* ctl) {
  __shared__ double sh[32];
  double m[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) m[a][b] = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    double x[D], y[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      x[k] = X[r * D + k];
      y[k] = Yv[r * D + k];
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) m[a][b] += y[a] * x[b];
  }
  double* part = s.partials + (long long)blockIdx.x * D * D;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const double v = block_sum(m[a][b], sh);
      if (threadIdx.x == 0) part[a * D + b] = v;
    }
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) {
      double M[D][D], Q[D][D];
      for (int o = 0; o < D * D; ++o) {
        double acc = 0.0;
        for (unsigned int bb = 0; bb < gridDim.x; ++bb) acc += s.partials[(long long)bb * D * D + o];
        M[o / D][o % D] = acc;
      }
      polar_fp64<D>(M, Q);
      for (int o = 0; o < D * D; ++o) s.Q[o] = Q[o / D][o % D];
      s.scal[1] = 0.0;
      ctl->counter = 0u;
    }
  }
}

template <int D>
__global__ void __launch_bounds__(256) dist_kernel(const float* __restrict__ X, const float* __restrict__ Yv,
                                                   long long rows, SpecScratch s, Ctl* ctl) {
  __shared__ double sh[32];
  __shared__ double q[D * D];
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) q[o] = s.Q[o];
  __syncthreads();
  double acc = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    double y[D];
#pragma unroll
    for (int k = 0; k < D; ++k) y[k] = Yv[r * D + k];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double yq = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) yq += y[k] * q[k * D + c];
      const double e = (double)X[r * D + c] - yq;
      acc += e * e;
    }
  }
  const double bs = block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(&s.scal[1], bs);
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) ctl->counter = 0u;
  }
}

// Copy the final iterate (in ping-pong buffer iters_done & 1) to the caller's X.
__global__ void copy_out_kernel(const float* __restrict__ X0, const float* __restrict__ X1, float* __restrict__ out,
                                long long count, const Ctl* ctl) {
  const float* src = (ctl->iters_done & 1) ? X1 : X0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = src[e];
}

// Spectral init's final basis sits in buffer spec_iters & 1 (the start V0 is in buffer 0
// after the initial orthonormalisation, which writes buffer 1 ... see host sequence).
__global__ void select_copy_kernel(const float* __restrict__ B0, const float* __restrict__ B1, float* __restrict__ out,
                                   long long count, const Ctl* ctl) {
  const float* src = (ctl->spec_iters & 1) ? B0 : B1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = src[e];
}

// ------------------------------------------------------------- dispatch
#define NSRGS_DISPATCH_D(d, F)        \
  switch (d) {                        \
    case 1: F(1); break;              \
    case 2: F(2); break;              \
    case 3: F(3); break;              \
    case 4: F(4); break;              \
    case 5: F(5); break;              \
    case 6: F(6); break;              \
    case 7: F(7); break;              \
    case 8: F(8); break;              \
    default: return cudaErrorInvalidValue; \
  }

// Runtime-d versions for 8 < d <= 64 (generic.cu).
cudaError_t launch_epilogue_generic(const float*, float*, float*, int, int, float, int, int, double, Ctl*, double*,
                                    cudaStream_t);
cudaError_t launch_spec_gram_generic(const float*, float*, float*, long long, int, float, int, int,
                                     const SpecScratch&, Ctl*, cudaStream_t);
cudaError_t launch_spec_update_generic(const float*, const float*, float*, long long, int, const SpecScratch&,
                                       double, int, Ctl*, cudaStream_t);
cudaError_t launch_polar_generic(const float*, float*, int, int, cudaStream_t);
cudaError_t launch_dF_generic(const float*, const float*, long long, int, const SpecScratch&, Ctl*, cudaStream_t);

cudaError_t launch_epilogue(const float* X, float* Y, float* Xout, int n, int d, float eta, int K, int safeguard,
                            double tol, Ctl* ctl, double* upd_out, cudaStream_t st) {
  if (d > kDmaxSmall) return launch_epilogue_generic(X, Y, Xout, n, d, eta, K, safeguard, tol, ctl, upd_out, st);
  const int grid = (n + 127) / 128;
#define L(DD) epilogue_kernel<DD><<<grid, 128, 0, st>>>(X, Y, Xout, n, eta, K, safeguard, tol, ctl, upd_out)
  NSRGS_DISPATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t launch_gpm_generic(const float*, float*, float*, int, int, double, Ctl*, cudaStream_t);

cudaError_t launch_gpm_epilogue(const float* X, float* Y, float* Xout, int n, int d, double tol, Ctl* ctl,
                                cudaStream_t st) {
  if (d > kDmaxSmall) return launch_gpm_generic(X, Y, Xout, n, d, tol, ctl, st);
  const int grid = (n + 127) / 128;
#define L(DD) gpm_epilogue_kernel<DD><<<grid, 128, 0, st>>>(X, Y, Xout, n, tol, ctl)
  NSRGS_DISPATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

int reduce_grid(long long rows) {
  long long g = (rows + 255) / 256;
  const long long cap = 2LL * num_sms();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_spec_v0(float* V, long long rows, int d, double* shift_slot, cudaStream_t st) {
  spec_v0_kernel<<<reduce_grid(rows), 256, 0, st>>>(V, rows, d, shift_slot);
  return cudaGetLastError();
}

// fp32: the chunk inner products in float32 (rounded-operand products, d > 8 only).
cudaError_t launch_spec_gram(const float* V, float* Y, float* W, long long rows, int d, float shift, int dev_shift,
                             int fp32, const SpecScratch& s, Ctl* ctl, cudaStream_t st) {
  if (d > kDmaxSmall) return launch_spec_gram_generic(V, Y, W, rows, d, shift, dev_shift, fp32, s, ctl, st);
  const int grid = reduce_grid(rows);
#define L(DD) spec_gram_kernel<DD><<<grid, 256, 0, st>>>(V, Y, W, rows, shift, dev_shift, s, ctl)
  NSRGS_DISPATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t launch_spec_update(const float* V, const float* W, float* Vnew, long long rows, int d,
                               const SpecScratch& s, double tol, int count_pass, Ctl* ctl, cudaStream_t st) {
  if (d > kDmaxSmall) return launch_spec_update_generic(V, W, Vnew, rows, d, s, tol, count_pass, ctl, st);
  const int grid = reduce_grid(rows);
#define L(DD) spec_update_kernel<DD><<<grid, 256, 0, st>>>(V, W, Vnew, rows, s, tol, count_pass, ctl)
  NSRGS_DISPATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t launch_polar_blocks(const float* V, float* X0, int n, int d, cudaStream_t st) {
  if (d > kDmaxSmall) return launch_polar_generic(V, X0, n, d, st);
  const int grid = (n + 127) / 128;
#define L(DD) polar_blocks_kernel<DD><<<grid, 128, 0, st>>>(V, X0, n)
  NSRGS_DISPATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t launch_dF(const float* X, const float* Yv, long long rows, int d, const SpecScratch& s, Ctl* ctl,
                      cudaStream_t st) {
  if (d > kDmaxSmall) return launch_dF_generic(X, Yv, rows, d, s, ctl, st);
  const int grid = reduce_grid(rows);
#define L(DD) cross_gram_kernel<DD><<<grid, 256, 0, st>>>(X, Yv, rows, s, ctl)
  NSRGS_DISPATCH_D(d, L)
#undef L
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
#define L(DD) dist_kernel<DD><<<grid, 256, 0, st>>>(X, Yv, rows, s, ctl)
  NSRGS_DISPATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t launch_copy_out(const float* X0, const float* X1, float* out, long long count, const Ctl* ctl,
                            cudaStream_t st) {
  copy_out_kernel<<<reduce_grid(count), 256, 0, st>>>(X0, X1, out, count, ctl);
  return cudaGetLastError();
}

cudaError_t launch_select_copy(const float* B0, const float* B1, float* out, long long count, const Ctl* ctl,
                               cudaStream_t st) {
  select_copy_kernel<<<reduce_grid(count), 256, 0, st>>>(B0, B1, out, count, ctl);
  return cudaGetLastError();
}

}  // namespace nsrgs

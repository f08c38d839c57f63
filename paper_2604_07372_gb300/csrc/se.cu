// SE(d) form (an extension §6 names; the paper writes no method for it): poses
// (X_i, t_i) with X_i in O(d) and t_i in R^d, measurements A_ij ~ X_i X_j^T and
// c_ij ~ X_i (t_j - t_i) for observed pairs i < j, objective
//     f(X, t) = F(X) + kappa sum_{i<j} w_ij ||t_j - t_i - X_i^T c_ij||^2.
// One iteration from (X^t, t^t), every block at once:
//     G^X_i = (n-1) X_i - sum_{j != i} A_ij X_j - kappa sum_{j>i} c_ij (t_j - t_i)^T
//     G^t_i = kappa [deg_i t_i - sum_{j~i} t_j - sum_{j<i} X_j^T c_ji + X_i^T sum_{j>i} c_ij]
//     X_i <- S_K(X_i - eta P_{X_i}(G^X_i))   (§2.2 projection, Algorithm 1)
//     t_i <- t_i - eta_t G^t_i.
// All pair sums come from one read of A: the packed matrix holds the augmented
// (d+1) x (d+1) blocks B_ij = [[A_ij, sqrt(kappa) c_ij], [0, w_ij]] (SeAugSrc) and
// the iterate the blocks Xa_j = [[X_j, 0], [sqrt(kappa) t_j^T, 1]], so the panel
// stream's Ya = B_off Xa holds, per block row i,
//     top-left  TL_i = sum_{j != i} A_ij X_j + kappa sum_{j>i} c_ij t_j^T
//     top-right TR_i = sqrt(kappa) sum_{j>i} c_ij
//     bottom-left BL_i = sqrt(kappa) (sum_{j~i} t_j + sum_{j<i} X_j^T c_ji)^T
//     bottom-right BR_i = deg_i,
// and G^X_i = (n-1) X_i - TL_i + sqrt(kappa) TR_i t_i^T,
//     G^t_i = kappa BR_i t_i - sqrt(kappa) BL_i^T + sqrt(kappa) X_i^T TR_i.
// The epilogue below is one thread per node, in registers, like the O(d) one, for
// d <= 7 (augmented blocks on the panel stream); for 8 <= d <= 63 a CTA per node
// with the d x d matrices in shared memory (augmented blocks in the tile layouts).
#include <math.h>

#include "blockops.cuh"

namespace nsrgs {

// Xa_i = [[X_i, 0], [sqrt(kappa) t_i^T, 1]] for every node.
template <int d>
__global__ void se_augment_kernel(const float* __restrict__ X, const float* __restrict__ t, float* __restrict__ Xa,
                                  int n, float sk) {
  constexpr int D = d + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long b = (long long)i * D * D;
#pragma unroll
  for (int r = 0; r < d; ++r) {
#pragma unroll
    for (int c = 0; c < d; ++c) Xa[b + r * D + c] = X[((long long)i * d + r) * d + c];
    Xa[b + r * D + d] = 0.f;
  }
#pragma unroll
  for (int c = 0; c < d; ++c) Xa[b + d * D + c] = sk * t[(long long)i * d + c];
  Xa[b + d * D + d] = 1.f;
}

// X_i = top-left d x d of the final augmented iterate (which of the two
// buffers holds it follows the iterations run).
template <int d>
__global__ void se_extract_kernel(const float* __restrict__ Xa0, const float* __restrict__ Xa1,
                                  float* __restrict__ X, int n, const Ctl* ctl) {
  constexpr int D = d + 1;
  const float* src = (ctl->iters_done & 1) ? Xa1 : Xa0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int r = 0; r < d; ++r)
#pragma unroll
    for (int c = 0; c < d; ++c) X[((long long)i * d + r) * d + c] = src[(long long)i * D * D + r * D + c];
}

template <int d>
__global__ void __launch_bounds__(128) se_epilogue_kernel(const float* __restrict__ Xa, float* __restrict__ Ya,
                                                          float* __restrict__ Xa_out, float* __restrict__ t, int n,
                                                          float eta, float eta_t, float kappa, int K, double tol,
                                                          Ctl* ctl) {
  constexpr int D = d + 1;
  __shared__ double sh[32];
  if (ctl->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double diff2 = 0.0;
  unsigned int flags = 0;
  if (i < n) {
    const float sk = sqrtf(kappa);
    const long long b = (long long)i * D * D;
    float x[d][d], y[D][D], ti[d];
#pragma unroll
    for (int r = 0; r < d; ++r)
#pragma unroll
      for (int c = 0; c < d; ++c) x[r][c] = Xa[b + r * D + c];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        y[r][c] = Ya[b + r * D + c];
        Ya[b + r * D + c] = 0.f;
      }
#pragma unroll
    for (int c = 0; c < d; ++c) ti[c] = t[(long long)i * d + c];
    // G^X = (n-1) X - TL + sqrt(kappa) TR t^T
    float gm[d][d];
    const float nm1 = (float)(n - 1);
#pragma unroll
    for (int r = 0; r < d; ++r)
#pragma unroll
      for (int c = 0; c < d; ++c) gm[r][c] = nm1 * x[r][c] - y[r][c] + sk * y[r][d] * ti[c];
    // G^t = kappa BR t - sqrt(kappa) BL^T + sqrt(kappa) X^T TR;  t' = t - eta_t G^t
    float tn[d];
#pragma unroll
    for (int c = 0; c < d; ++c) {
      float xtr = 0.f;
#pragma unroll
      for (int r = 0; r < d; ++r) xtr = fmaf(x[r][c], y[r][d], xtr);
      const float gt = kappa * y[d][d] * ti[c] - sk * y[d][c] + sk * xtr;
      tn[c] = ti[c] - eta_t * gt;
    }
    // F = X - eta (G - X G^T X) / 2
    float m[d][d];
#pragma unroll
    for (int r = 0; r < d; ++r)
#pragma unroll
      for (int c = 0; c < d; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < d; ++k) acc = fmaf(gm[k][r], x[k][c], acc);  // G^T X
        m[r][c] = acc;
      }
    float s[d][d];
    const float h = 0.5f * eta;
#pragma unroll
    for (int r = 0; r < d; ++r)
#pragma unroll
      for (int c = 0; c < d; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < d; ++k) acc = fmaf(x[r][k], m[k][c], acc);
        s[r][c] = x[r][c] - h * (gm[r][c] - acc);
      }
    {  // Lemma 2.1 precondition, checked with ||I - F^T F||_F
      float e2 = 0.f;
#pragma unroll
      for (int r = 0; r < d; ++r)
#pragma unroll
        for (int c = 0; c < d; ++c) {
          float acc = (r == c) ? 1.f : 0.f;
#pragma unroll
          for (int k = 0; k < d; ++k) acc = fmaf(-s[k][r], s[k][c], acc);
          e2 = fmaf(acc, acc, e2);
        }
      if (!(e2 < 1.f)) flags |= FLAG_NS_PRECOND;
    }
    for (int k = 0; k < K; ++k) {  // Algorithm 1: S <- S (3I - S^T S) / 2
#pragma unroll
      for (int r = 0; r < d; ++r)
#pragma unroll
        for (int c = 0; c < d; ++c) {
          float acc = (r == c) ? 3.f : 0.f;
#pragma unroll
          for (int l = 0; l < d; ++l) acc = fmaf(-s[l][r], s[l][c], acc);
          m[r][c] = acc;
        }
      float sn[d][d];
#pragma unroll
      for (int r = 0; r < d; ++r)
#pragma unroll
        for (int c = 0; c < d; ++c) {
          float acc = 0.f;
#pragma unroll
          for (int l = 0; l < d; ++l) acc = fmaf(s[r][l], m[l][c], acc);
          sn[r][c] = 0.5f * acc;
        }
#pragma unroll
      for (int r = 0; r < d; ++r)
#pragma unroll
        for (int c = 0; c < d; ++c) s[r][c] = sn[r][c];
    }
    bool finite = true;
#pragma unroll
    for (int r = 0; r < d; ++r) {
#pragma unroll
      for (int c = 0; c < d; ++c) {
        const float v = s[r][c];
        finite = finite && isfinite(v);
        Xa_out[b + r * D + c] = v;
        const double dd = (double)v - (double)x[r][c];
        diff2 += dd * dd;
      }
      Xa_out[b + r * D + d] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < d; ++c) {
      finite = finite && isfinite(tn[c]);
      Xa_out[b + d * D + c] = sk * tn[c];
      t[(long long)i * d + c] = tn[c];
      const double dd = (double)tn[c] - (double)ti[c];
      diff2 += dd * dd;
    }
    Xa_out[b + d * D + d] = 1.f;
    if (!finite) flags |= FLAG_NONFINITE;
  }
  if (flags) atomicOr(&ctl->flags, flags);
  const double bs = block_sum(diff2, sh);
  if (threadIdx.x == 0) atomicAdd(&ctl->upd_acc, bs);
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) {
      const double tot = atomicAdd(&ctl->upd_acc, 0.0);
      const double un = sqrt(tot / ((double)n * d));
      ctl->last_upd = un;
      ctl->iters_done += 1;
      if (tol > 0.0 && un < tol) ctl->stop = 1;
      ctl->upd_acc = 0.0;
      ctl->counter = 0u;
    }
  }
}

template <int d>
static cudaError_t se_launch_d(int what, const float* X, float* t, const float* Xa0, float* Ya, float* Xa1, int n,
                               float eta, float eta_t, float kappa, int K, double tol, Ctl* ctl, float* Xout,
                               cudaStream_t st) {
  const int grid = (n + 127) / 128;
  if (what == 0)
    se_augment_kernel<d><<<grid, 128, 0, st>>>(X, t, Xa1, n, sqrtf(kappa));
  else if (what == 1)
    se_epilogue_kernel<d><<<grid, 128, 0, st>>>(Xa0, Ya, Xa1, t, n, eta, eta_t, kappa, K, tol, ctl);
  else
    se_extract_kernel<d><<<grid, 128, 0, st>>>(Xa0, Xa1, Xout, n, ctl);
  return cudaGetLastError();
}

// ------------------------------------------------------- d >= 8 (runtime d)
// The same three steps with the d x d matrices in shared memory, one CTA per
// node (d + 1 = D up to 64; the augmented blocks then sit in the tile layouts).
__global__ void __launch_bounds__(256) se_augment_generic_kernel(const float* __restrict__ X,
                                                                 const float* __restrict__ t, float* __restrict__ Xa,
                                                                 int n, int d, float sk) {
  const int D = d + 1;
  const long long total = (long long)n * D * D;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / (D * D);
    const int r = (int)(e % (D * D)) / D, c = (int)(e % D);
    float v;
    if (r < d) v = c < d ? X[(i * d + r) * d + c] : 0.f;
    else v = c < d ? sk * t[i * d + c] : 1.f;
    Xa[e] = v;
  }
}

__global__ void __launch_bounds__(256) se_extract_generic_kernel(const float* __restrict__ Xa0,
                                                                 const float* __restrict__ Xa1,
                                                                 float* __restrict__ X, int n, int d,
                                                                 const Ctl* ctl) {
  const int D = d + 1;
  const float* src = (ctl->iters_done & 1) ? Xa1 : Xa0;
  const long long total = (long long)n * d * d;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / (d * d);
    const int r = (int)(e % (d * d)) / d, c = (int)(e % d);
    X[e] = src[i * D * D + r * D + c];
  }
}

// Row-major d x d products in shared memory: C = op(A) B (C distinct from A, B).
__device__ static void se_mm(const float* A, bool transA, const float* B, float* C, int d) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int r = e / d, c = e % d;
    float acc = 0.f;
    for (int k = 0; k < d; ++k) acc = fmaf(transA ? A[k * d + r] : A[r * d + k], B[k * d + c], acc);
    C[e] = acc;
  }
}

// Dynamic shared memory: 5 d x d floats (x, g, m, s, u) and 2 d floats (t, t').
__global__ void __launch_bounds__(256) se_epilogue_generic_kernel(const float* __restrict__ Xa,
                                                                  float* __restrict__ Ya,
                                                                  float* __restrict__ Xa_out, float* __restrict__ t,
                                                                  int n, int d, float eta, float eta_t, float kappa,
                                                                  int K, double tol, Ctl* ctl) {
  extern __shared__ __align__(16) float sse[];
  __shared__ double sh[32];
  __shared__ unsigned int s_flags;
  if (ctl->stop) return;
  const int D = d + 1, dd = d * d;
  const long long i = blockIdx.x, b = i * D * D;
  float* x = sse;
  float* g = x + dd;
  float* m = g + dd;
  float* sm = m + dd;
  float* u = sm + dd;
  float* ti = u + dd;
  float* tn = ti + d;
  const float sk = sqrtf(kappa), nm1 = (float)(n - 1);
  if (threadIdx.x == 0) s_flags = 0u;
  for (int e = threadIdx.x; e < d; e += blockDim.x) ti[e] = t[i * d + e];
  __syncthreads();
  // G^X = (n-1) X - TL + sqrt(kappa) TR t^T   (Y read, then cleared for the next pass)
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, c = e % d;
    x[e] = Xa[b + r * D + c];
    g[e] = nm1 * x[e] - Ya[b + r * D + c] + sk * Ya[b + r * D + d] * ti[c];
  }
  // G^t = kappa BR t - sqrt(kappa) BL^T + sqrt(kappa) X^T TR;  t' = t - eta_t G^t
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    float xtr = 0.f;
    for (int r = 0; r < d; ++r) xtr = fmaf(x[r * d + c], Ya[b + r * D + d], xtr);
    const float gt = kappa * Ya[b + d * D + d] * ti[c] - sk * Ya[b + d * D + c] + sk * xtr;
    tn[c] = ti[c] - eta_t * gt;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) Ya[b + e] = 0.f;
  // F = X - eta (G - X G^T X) / 2
  se_mm(g, true, x, m, d);  // G^T X
  __syncthreads();
  se_mm(x, false, m, u, d);  // X G^T X
  __syncthreads();
  const float h = 0.5f * eta;
  for (int e = threadIdx.x; e < dd; e += blockDim.x) sm[e] = x[e] - h * (g[e] - u[e]);
  __syncthreads();
  // Lemma 2.1 precondition, checked with ||I - F^T F||_F
  se_mm(sm, true, sm, m, d);
  __syncthreads();
  double e2 = 0.0;
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const double v = ((e / d == e % d) ? 1.0 : 0.0) - (double)m[e];
    e2 += v * v;
  }
  e2 = block_sum(e2, sh);
  if (threadIdx.x == 0 && !(e2 < 1.0)) s_flags |= FLAG_NS_PRECOND;
  for (int k = 0; k < K; ++k) {  // Algorithm 1: S <- S (3I - S^T S) / 2
    __syncthreads();
    se_mm(sm, true, sm, m, d);
    __syncthreads();
    for (int e = threadIdx.x; e < dd; e += blockDim.x) m[e] = ((e / d == e % d) ? 3.f : 0.f) - m[e];
    __syncthreads();
    se_mm(sm, false, m, u, d);
    __syncthreads();
    for (int e = threadIdx.x; e < dd; e += blockDim.x) sm[e] = 0.5f * u[e];
  }
  __syncthreads();
  double diff2 = 0.0;
  bool finite = true;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    float v;
    if (r < d && c < d) {
      v = sm[r * d + c];
      const double q = (double)v - (double)x[r * d + c];
      diff2 += q * q;
      finite = finite && isfinite(v);
    } else if (r < d) {
      v = 0.f;
    } else if (c < d) {
      v = sk * tn[c];
      const double q = (double)tn[c] - (double)ti[c];
      diff2 += q * q;
      finite = finite && isfinite(tn[c]);
      t[i * d + c] = tn[c];
    } else {
      v = 1.f;
    }
    Xa_out[b + e] = v;
  }
  if (!finite) atomicOr(&s_flags, FLAG_NONFINITE);
  const double bs = block_sum(diff2, sh);
  if (threadIdx.x == 0) {
    if (s_flags) atomicOr(&ctl->flags, s_flags);
    atomicAdd(&ctl->upd_acc, bs);
  }
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0) {
      const double tot = atomicAdd(&ctl->upd_acc, 0.0);
      const double un = sqrt(tot / ((double)n * d));
      ctl->last_upd = un;
      ctl->iters_done += 1;
      if (tol > 0.0 && un < tol) ctl->stop = 1;
      ctl->upd_acc = 0.0;
      ctl->counter = 0u;
    }
  }
}

static size_t se_generic_smem(int d) { return (size_t)(5 * d * d + 2 * d) * sizeof(float); }

cudaError_t se_prepare(int d) {
  if (d <= 7) return cudaSuccess;
  return cudaFuncSetAttribute(se_epilogue_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)se_generic_smem(d));
}

// what: 0 = augment (X, t -> Xa1), 1 = epilogue (Xa0, Ya -> Xa1, t), 2 = extract
// (Xa0 / Xa1 -> Xout by the iterations run).  d in 1..63 (register kernels up to 7).
cudaError_t se_launch(int what, int d, const float* X, float* t, const float* Xa0, float* Ya, float* Xa1, int n,
                      float eta, float eta_t, float kappa, int K, double tol, Ctl* ctl, float* Xout,
                      cudaStream_t st) {
  switch (d) {
    case 1: return se_launch_d<1>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
    case 2: return se_launch_d<2>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
    case 3: return se_launch_d<3>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
    case 4: return se_launch_d<4>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
    case 5: return se_launch_d<5>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
    case 6: return se_launch_d<6>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
    case 7: return se_launch_d<7>(what, X, t, Xa0, Ya, Xa1, n, eta, eta_t, kappa, K, tol, ctl, Xout, st);
  }
  if (d < 8 || d > 63) return cudaErrorInvalidValue;
  const int grid = 4 * num_sms();
  if (what == 0)
    se_augment_generic_kernel<<<grid, 256, 0, st>>>(X, t, Xa1, n, d, sqrtf(kappa));
  else if (what == 1)
    se_epilogue_generic_kernel<<<n, 256, se_generic_smem(d), st>>>(Xa0, Ya, Xa1, t, n, d, eta, eta_t, kappa, K,
                                                                   tol, ctl);
  else
    se_extract_generic_kernel<<<grid, 256, 0, st>>>(Xa0, Xa1, Xout, n, d, ctl);
  return cudaGetLastError();
}

}  // namespace nsrgs

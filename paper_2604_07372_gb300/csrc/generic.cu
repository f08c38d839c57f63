// Per-block d x d work for block sizes above 8 (runtime d <= 64): one CTA per
// block with the d x d matrices in shared memory.  Same arithmetic as the
// register kernels of small.cu:
//   * iteration epilogue (Algorithm 2's loop body, §2.2 projection, Algorithm 1);
//   * spectral subspace step (float64 Gram / Cholesky / V <- W R^{-1} / residual);
//   * exact blockwise sign for X^0 and for d_F: Newton-Schulz run to convergence in
//     float64 on M / ||M||_F (all singular values in (0, 1], so the iteration
//     converges to the polar factor U V^T of any full-rank M);
//   * d_F(X, Y) (§1.4).
#include <math.h>

#include <type_traits>

#include "blockops.cuh"

namespace nsrgs {

// C = alpha * op(A) * B + beta * C0 for D x D row-major matrices in shared memory
// (op(A) = A or A^T).  Each thread owns TS x TS tiles of C, TS the largest of 4, 2,
// 1 that still gives every thread of the CTA a tile (one 4 x 4 tile per thread at
// D = 64: a k step costs 8 shared loads for 16 FMAs); C must not alias A or B.
template <typename T, int TS>
__device__ void cta_mm_ts(const T* A, bool transA, const T* B, T* C, int D, T alpha, const T* C0, T beta) {
  const int tn = (D + TS - 1) / TS, tiles = tn * tn;
  for (int tt = threadIdx.x; tt < tiles; tt += blockDim.x) {
    const int r0 = (tt / tn) * TS, c0 = (tt % tn) * TS;
    T acc[TS][TS];
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j) acc[i][j] = 0;
    for (int k = 0; k < D; ++k) {
      T a[TS], b[TS];
#pragma unroll
      for (int i = 0; i < TS; ++i) {
        const int r = r0 + i, c = c0 + i;
        a[i] = r < D ? (transA ? A[k * D + r] : A[r * D + k]) : T(0);
        b[i] = c < D ? B[k * D + c] : T(0);
      }
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) acc[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j) {
        const int r = r0 + i, c = c0 + j;
        if (r < D && c < D) C[r * D + c] = alpha * acc[i][j] + (C0 ? beta * C0[r * D + c] : T(0));
      }
  }
}

template <typename T>
__device__ void cta_mm(const T* A, bool transA, const T* B, T* C, int D, T alpha, const T* C0, T beta) {
  if (D * D >= 16 * (int)blockDim.x)
    cta_mm_ts<T, 4>(A, transA, B, C, D, alpha, C0, beta);
  else if (D * D >= 4 * (int)blockDim.x)
    cta_mm_ts<T, 2>(A, transA, B, C, D, alpha, C0, beta);
  else
    cta_mm_ts<T, 1>(A, transA, B, C, D, alpha, C0, beta);
}

// ------------------------------------------------------------ epilogue
// Dynamic shared memory: 5 D x D float matrices.
__global__ void __launch_bounds__(256) epilogue_generic_kernel(const float* __restrict__ X, float* __restrict__ Y,
                                                               float* __restrict__ Xout, int n, int D, float eta,
                                                               int K, int safeguard, double tol, Ctl* ctl,
                                                               double* upd_out) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double sh[32];
  if (ctl->stop) return;
  const int DD = D * D;
  float* x = sm;
  float* g = sm + DD;
  float* t = sm + 2 * DD;
  float* s = sm + 3 * DD;
  float* m = sm + 4 * DD;
  const long long base = (long long)blockIdx.x * DD;
  const float nm1 = (float)(n - 1);
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    x[e] = X[base + e];
    g[e] = nm1 * x[e] - Y[base + e];
    Y[base + e] = 0.f;
  }
  __syncthreads();
  cta_mm<float>(g, true, x, t, D, 1.f, nullptr, 0.f);  // t = G^T X
  __syncthreads();
  cta_mm<float>(x, false, t, m, D, 1.f, nullptr, 0.f);  // m = X G^T X
  __syncthreads();
  for (int e = threadIdx.x; e < DD; e += blockDim.x) s[e] = x[e] - 0.5f * eta * (g[e] - m[e]);  // F
  __syncthreads();
  // Lemma 2.1 precondition (||I - F^T F||_F >= 1 flags it)
  cta_mm<float>(s, true, s, m, D, 1.f, nullptr, 0.f);
  __syncthreads();
  double e2 = 0.0;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    const double v = ((e / D == e % D) ? 1.0 : 0.0) - (double)m[e];
    e2 += v * v;
  }
  e2 = block_sum(e2, sh);
  __shared__ double fnorm;
  if (threadIdx.x == 0) fnorm = !(e2 < 1.0) ? 1.0 : 0.0;  // 1: precondition fails
  __syncthreads();
  if (fnorm != 0.0) {
    if (safeguard) {
      // safeguarded start (beyond the paper): F / ||F||_F, same polar factor
      double f2 = 0.0;
      for (int e = threadIdx.x; e < DD; e += blockDim.x) f2 += (double)s[e] * (double)s[e];
      f2 = block_sum(f2, sh);
      __syncthreads();
      if (threadIdx.x == 0) {
        fnorm = sqrt(f2);
        atomicOr(&ctl->flags, FLAG_NS_SAFEGUARDED);
      }
      __syncthreads();
      const float inv = (float)(1.0 / fnorm);
      for (int e = threadIdx.x; e < DD; e += blockDim.x) s[e] *= inv;
    } else if (threadIdx.x == 0) {
      atomicOr(&ctl->flags, FLAG_NS_PRECOND);
    }
  }
  for (int k = 0; k < K; ++k) {
    __syncthreads();
    cta_mm<float>(s, true, s, m, D, 1.f, nullptr, 0.f);  // S^T S
    __syncthreads();
    for (int e = threadIdx.x; e < DD; e += blockDim.x) m[e] = ((e / D == e % D) ? 3.f : 0.f) - m[e];
    __syncthreads();
    cta_mm<float>(s, false, m, g, D, 0.5f, nullptr, 0.f);  // S (3I - S^T S) / 2
    __syncthreads();
    for (int e = threadIdx.x; e < DD; e += blockDim.x) s[e] = g[e];
  }
  __syncthreads();
  double diff2 = 0.0;
  bool finite = true;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    finite = finite && isfinite(s[e]);
    Xout[base + e] = s[e];
    const double dd = (double)s[e] - (double)x[e];
    diff2 += dd * dd;
  }
  if (!finite) atomicOr(&ctl->flags, FLAG_NONFINITE);
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

// ---------------------------------------------- GPM (comparison method)
// Generalised power method step for 8 < d <= 64, CTA per block: M = Y_i + X_i,
// X_i <- sgn(M) by a float32 one-sided Jacobi SVD (the batched per-block SVD
// that the comparison method pays for every iteration).  The columns of M are
// paired round-robin: d/2 disjoint pairs per round (a dummy column when d is
// odd), one warp per pair, d - 1 rounds per sweep, sweeps until every pair is
// orthogonal to 1e-6 (at most 20).  Then U = M V with unit columns and
// sgn(M) = U V^T.  Shared memory: U and V (column-major) and X_i, 3 D x D
// floats.  Same update-norm / stop bookkeeping as the epilogue.
__global__ void __launch_bounds__(256) gpm_generic_kernel(const float* __restrict__ X, float* __restrict__ Y,
                                                          float* __restrict__ Xout, int n, int D, double tol,
                                                          Ctl* ctl) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double sh[32];
  __shared__ float woff[8];
  if (ctl->stop) return;
  const int DD = D * D;
  float* U = sm;           // column c at U + c * D
  float* Vm = sm + DD;     // column c at Vm + c * D
  float* x = sm + 2 * DD;  // X_i, row-major
  const long long base = (long long)blockIdx.x * DD;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    const int r = e / D, c = e % D;
    const float xv = X[base + e];
    x[e] = xv;
    U[c * D + r] = Y[base + e] + xv;
    Y[base + e] = 0.f;
    Vm[c * D + r] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
  const int m = D + (D & 1);  // columns in the round-robin, with a dummy when D is odd
  for (int sweep = 0; sweep < 20; ++sweep) {
    float off = 0.f;  // warp-uniform
    for (int rd = 0; rd < m - 1; ++rd) {
      for (int k = warp; k < m / 2; k += nw) {
        int p, q;
        if (k == 0) {
          p = m - 1;
          q = rd;
        } else {
          p = (rd + k) % (m - 1);
          q = (rd - k + (m - 1)) % (m - 1);
        }
        if (p >= D || q >= D) continue;
        float* up = U + p * D;
        float* uq = U + q * D;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int r = lane; r < D; r += 32) {
          al = fmaf(up[r], up[r], al);
          be = fmaf(uq[r], uq[r], be);
          ga = fmaf(up[r], uq[r], ga);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        const float nrm = sqrtf(al * be);
        if (nrm == 0.f || fabsf(ga) <= 1e-8f * nrm) continue;
        off = fmaxf(off, fabsf(ga) / nrm);
        const float zeta = (be - al) / (2.f * ga);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float c = rsqrtf(1.f + t * t);
        const float sn = c * t;
        float* vp = Vm + p * D;
        float* vq = Vm + q * D;
        for (int r = lane; r < D; r += 32) {
          const float a1 = up[r], a2 = uq[r];
          up[r] = c * a1 - sn * a2;
          uq[r] = sn * a1 + c * a2;
          const float b1 = vp[r], b2 = vq[r];
          vp[r] = c * b1 - sn * b2;
          vq[r] = sn * b1 + c * b2;
        }
      }
      __syncthreads();
    }
    if (lane == 0) woff[warp] = off;
    __syncthreads();
    float mo = 0.f;
    for (int w = 0; w < nw; ++w) mo = fmaxf(mo, woff[w]);
    __syncthreads();
    if (mo < 1e-6f) break;
  }
  for (int c = warp; c < D; c += nw) {  // unit columns: U_svd = M V Sigma^{-1}
    float s2 = 0.f;
    for (int r = lane; r < D; r += 32) s2 = fmaf(U[c * D + r], U[c * D + r], s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const float inv = s2 > 0.f ? rsqrtf(s2) : 0.f;
    for (int r = lane; r < D; r += 32) U[c * D + r] *= inv;
  }
  __syncthreads();
  double diff2 = 0.0;
  bool finite = true;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    const int r = e / D, c = e % D;
    float q = 0.f;
    for (int k = 0; k < D; ++k) q = fmaf(U[k * D + r], Vm[k * D + c], q);
    finite = finite && isfinite(q);
    Xout[base + e] = q;
    const double dd = (double)q - (double)x[e];
    diff2 += dd * dd;
  }
  if (!finite) atomicOr(&ctl->flags, FLAG_NONFINITE);
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

// ------------------------------------------------- exact sign (float64)
// S <- M / ||M||_F, then S <- S (3I - S^T S)/2 until ||I - S^T S||_F < 1e-14.  The
// iterations far from the polar factor run in float32 (GB300's float64 pipe is a
// small fraction of its float32 one) until ||I - S^T S||_F < 1e-4; the quadratic
// convergence then takes the float64 iterations from there to rounding level in
// two or three steps.  Shared scratch: 3 D x D doubles (S, T, U) and 3 D x D floats
// (Sf, Tf, Uf).  Result in S.
__device__ void cta_polar_ns64(const double* M, double* S, double* T, double* U, float* Sf, float* Tf, float* Uf,
                               int D, double* sh) {
  const int DD = D * D;
  double f2 = 0.0;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) f2 += M[e] * M[e];
  f2 = block_sum(f2, sh);
  __shared__ double s_norm;
  __shared__ int s_done;
  if (threadIdx.x == 0) s_norm = f2 > 0.0 ? 1.0 / sqrt(f2) : 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < DD; e += blockDim.x) Sf[e] = (float)(M[e] * s_norm);
  for (int it = 0; it < 100; ++it) {
    __syncthreads();
    cta_mm<float>(Sf, true, Sf, Tf, D, 1.f, nullptr, 0.f);  // S^T S
    __syncthreads();
    double err = 0.0;
    for (int e = threadIdx.x; e < DD; e += blockDim.x) {
      const float v = ((e / D == e % D) ? 1.f : 0.f) - Tf[e];
      err += (double)v * v;
      Tf[e] = ((e / D == e % D) ? 3.f : 0.f) - Tf[e];
    }
    err = block_sum(err, sh);
    if (threadIdx.x == 0) s_done = err < 1e-8;
    __syncthreads();
    if (s_done) break;
    cta_mm<float>(Sf, false, Tf, Uf, D, 0.5f, nullptr, 0.f);
    __syncthreads();
    for (int e = threadIdx.x; e < DD; e += blockDim.x) Sf[e] = Uf[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < DD; e += blockDim.x) S[e] = (double)Sf[e];
  for (int it = 0; it < 100; ++it) {
    __syncthreads();
    cta_mm<double>(S, true, S, T, D, 1.0, nullptr, 0.0);  // S^T S
    __syncthreads();
    double err = 0.0;
    for (int e = threadIdx.x; e < DD; e += blockDim.x) {
      const double v = ((e / D == e % D) ? 1.0 : 0.0) - T[e];
      err += v * v;
      T[e] = ((e / D == e % D) ? 3.0 : 0.0) - T[e];
    }
    err = block_sum(err, sh);
    // converged to rounding level (a few ulps times d), or out of iterations
    if (threadIdx.x == 0) s_done = (err < 16.0 * D * D * 4.9e-32) || (it == 99);
    __syncthreads();
    if (s_done) break;
    cta_mm<double>(S, false, T, U, D, 0.5, nullptr, 0.0);
    __syncthreads();
    for (int e = threadIdx.x; e < DD; e += blockDim.x) S[e] = U[e];
  }
  __syncthreads();
}

// X0_i = sgn(V_i), CTA per block.  Dynamic shared memory: 4 D x D doubles, 3 D x D floats.
__global__ void __launch_bounds__(256) polar_generic_kernel(const float* __restrict__ V, float* __restrict__ X0, int D) {
  extern __shared__ __align__(16) double smd[];
  __shared__ double sh[32];
  const int DD = D * D;
  double* M = smd;
  float* f = reinterpret_cast<float*>(smd + 4 * DD);
  const long long base = (long long)blockIdx.x * DD;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) M[e] = V[base + e];
  __syncthreads();
  cta_polar_ns64(M, smd + DD, smd + 2 * DD, smd + 3 * DD, f, f + DD, f + 2 * DD, D, sh);
  for (int e = threadIdx.x; e < DD; e += blockDim.x) X0[base + e] = (float)smd[DD + e];
}

// ----------------------------------------------------- Gram reductions
// Partial sums over chunks of rows of P^T Q (and, in the spectral mode, first
// W = Y + shift V, then P = Q = W and a second product V^T W).
// Outputs: (P^T Q)[a][b] (mode 0: W^T W into s.WW; mode 1: Yv^T Xq into s.M) and, in
// mode 0, (V^T W)[a][b] into s.H.
// A chunk of 64 rows is staged in shared memory (as T, columns padded to DP, a
// multiple of 8); each thread owns a 4 x 8 tile of one product's outputs, so a
// row of the chunk costs it 12 shared loads for 32 FMAs.  T: the arithmetic of the
// inner products (float64; float32 for the tensor-core storages, whose residual
// floor sits near 1e-3: then a CTA sums its rows in float32 and the CTAs' sums
// are added in float64).
constexpr int kRowsPerCta = 64;

template <typename T>
__global__ void __launch_bounds__(256) gram_generic_kernel(const float* __restrict__ V, float* __restrict__ Yv,
                                                           float* __restrict__ W, const float* __restrict__ Xq,
                                                           long long rows, int D, float shift, int dev_shift,
                                                           int mode, SpecScratch s, Ctl* ctl) {
  extern __shared__ __align__(16) double smg_raw[];
  T* smg = reinterpret_cast<T*>(smg_raw);
  if (mode == 0 && ctl->spec_skip) return;
  // spectral mode: W = Y + c V, c the orthonormalising pass's `shift` or the current
  // shift; a restart pass (after a failed algebraic top-d test) takes W = V^0
  const bool restart = mode == 0 && dev_shift && ctl->spec_restart;
  const float c = (mode == 0 && dev_shift) ? (float)s.scal[3] : shift;
  const int DD = D * D;
  const int DP = (D + 7) & ~7;
  const int nprod = mode == 0 ? 2 : 1;
  T* Pm = smg;                    // kRowsPerCta x DP: V (mode 0) or Yv (mode 1)
  T* Qm = smg + kRowsPerCta * DP; // kRowsPerCta x DP: W (mode 0) or Xq (mode 1)
  // thread -> (product g, 4-row block ta, 8-column block tb)
  const int tb_n = DP / 8, tiles = (DP / 4) * tb_n;
  const int g = threadIdx.x / tiles, rem = threadIdx.x % tiles;
  const bool active = g < nprod;
  const int a0 = (rem / tb_n) * 4, b0 = (rem % tb_n) * 8;
  // mode 0: g = 0 -> W^T W (P = Q = W), g = 1 -> V^T W; mode 1: Yv^T Xq
  const T* Pg = (mode == 0 && g == 0) ? Qm : Pm;
  double acc[4][8];
  float accf[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0, accf[i][j] = 0.f;
  for (long long r0 = (long long)blockIdx.x * kRowsPerCta; r0 < rows; r0 += (long long)gridDim.x * kRowsPerCta) {
    const int nr = (int)min((long long)kRowsPerCta, rows - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * D; e += blockDim.x) {
      const long long ge = r0 * D + e;
      const int si = (e / D) * DP + e % D;
      if (mode == 0) {
        const float v = V[ge];
        const float w = restart ? spec_v0_entry(ge) : Yv[ge] + c * v;
        W[ge] = w;
        Yv[ge] = 0.f;
        Pm[si] = (T)v;
        Qm[si] = (T)w;
      } else {
        Pm[si] = (T)Yv[ge];
        Qm[si] = (T)Xq[ge];
      }
    }
    __syncthreads();
    if constexpr (std::is_same<T, double>::value) {  // float64: straight into the totals
      if (!active) continue;
      for (int r = 0; r < nr; ++r) {
        double p[4], q[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = (double)Pg[r * DP + a0 + i];
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = (double)Qm[r * DP + b0 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] += p[i] * q[j];
      }
    } else {
      // float32: the whole CTA range in float32 registers (a few thousand rows at
      // most, ~1e-6 relative against a residual floor near 1e-3)
      if (!active) continue;
      for (int r = 0; r < nr; ++r) {
        float p[4], q[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = (float)Pg[r * DP + a0 + i];
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = (float)Qm[r * DP + b0 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) accf[i][j] += p[i] * q[j];
      }
    }
  }
  const int nout = nprod * DD;
  double* part = s.partials + (long long)blockIdx.x * nout;
  if (active) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (a0 + i < D && b0 + j < D)
          part[g * DD + (a0 + i) * D + b0 + j] = std::is_same<T, double>::value ? acc[i][j] : (double)accf[i][j];
  }
}

// The CTAs' partial sums of gram_generic_kernel added up (thread per output,
// coalesced over the partials), then, by the last CTA: mode 0 ||H||_F^2 and the
// Cholesky factor of W^T W with its inverse (R^T R = W^T W, all threads of the
// CTA; R^{-1} by columns), mode 1 nothing more.  Dynamic shared memory: D x D doubles.
__global__ void __launch_bounds__(256) gram_finish_kernel(int nparts, int D, int mode, SpecScratch s, Ctl* ctl) {
  extern __shared__ __align__(16) double smf[];
  __shared__ double sh[32];
  if (mode == 0 && ctl->spec_skip) return;
  const int DD = D * D, nout = (mode == 0 ? 2 : 1) * DD;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < nout) {
    double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int b = 0;
    for (; b + 8 <= nparts; b += 8)
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] += s.partials[(long long)(b + u) * nout + o];
    for (; b < nparts; ++b) t[0] += s.partials[(long long)b * nout + o];
    const double a = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    if (mode == 0) {
      if (o < DD) s.WW[o] = a; else s.H[o - DD] = a;
    } else {
      s.M[o] = a;
    }
  }
  if (!last_block(&ctl->counter)) return;
  if (mode != 0) {
    if (threadIdx.x == 0) {
      s.scal[1] = 0.0;
      ctl->counter = 0u;
    }
    return;
  }
  double h2 = 0.0;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) h2 += s.H[e] * s.H[e];
  h2 = block_sum(h2, sh);
  // right-looking Cholesky in shared memory: row j of R = A[j][j..] after step j
  double* A = smf;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) A[e] = s.WW[e];
  __syncthreads();
  for (int j = 0; j < D; ++j) {
    if (threadIdx.x == 0) A[j * D + j] = sqrt(fmax(A[j * D + j], 1e-300));
    __syncthreads();
    const double rjj = A[j * D + j];
    for (int i = j + 1 + threadIdx.x; i < D; i += blockDim.x) A[j * D + i] /= rjj;
    __syncthreads();
    const int m = D - j - 1;  // trailing block rows/columns j+1 .. D-1, upper part
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = j + 1 + e / m, c = j + 1 + e % m;
      if (c >= r) A[r * D + c] -= A[j * D + r] * A[j * D + c];
    }
    __syncthreads();
  }
  // R^{-1} (upper triangular) by back substitution, one column per thread
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    for (int r = D - 1; r >= 0; --r) {
      double t = (r == c) ? 1.0 : 0.0;
      for (int k = r + 1; k <= c; ++k) t -= A[r * D + k] * s.Rinv[k * D + c];
      s.Rinv[r * D + c] = (r <= c) ? t / A[r * D + r] : 0.0;
    }
  }
  if (threadIdx.x == 0) {
    s.scal[0] = h2;
    s.scal[2] = 0.0;
    ctl->counter = 0u;
  }
}

// Vnew = W Rinv and the residual ||W - V H||^2 (thread per row); the last CTA
// finishes ||A V - V H||_F / ||H||_F.  Dynamic shared memory: Rinv and H (as T;
// T as in gram_generic_kernel, the residual summed in float64).
template <typename T>
__global__ void __launch_bounds__(256) update_generic_kernel(const float* __restrict__ V, const float* __restrict__ W,
                                                             float* __restrict__ Vnew, long long rows, int D,
                                                             SpecScratch s, double tol, int count_pass, Ctl* ctl) {
  extern __shared__ __align__(16) double smu_raw[];
  __shared__ double sh[32];
  if (ctl->spec_skip) return;
  const int DD = D * D;
  T* rinv = reinterpret_cast<T*>(smu_raw);
  T* hh = rinv + DD;
  for (int o = threadIdx.x; o < DD; o += blockDim.x) {
    rinv[o] = (T)s.Rinv[o];
    hh[o] = (T)s.H[o];
  }
  __syncthreads();
  // Columns in tiles of 16 with k outer, so each row element is converted to
  // float64 once per tile (float64 conversions share GB300's slow float64 pipe);
  // every sum keeps its order over k.
  constexpr int kTile = 16;
  double res = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
    const float* w = W + r * D;
    const float* v = V + r * D;
    for (int c0 = 0; c0 < D; c0 += kTile) {
      T nv[kTile], vh[kTile];
#pragma unroll
      for (int j = 0; j < kTile; ++j) nv[j] = vh[j] = 0;
      for (int k = 0; k < D; ++k) {
        const T wk = w[k], vk = v[k];
#pragma unroll
        for (int j = 0; j < kTile; ++j)
          if (c0 + j < D) {
            nv[j] += wk * rinv[k * D + c0 + j];
            vh[j] += vk * hh[k * D + c0 + j];
          }
      }
#pragma unroll
      for (int j = 0; j < kTile; ++j)
        if (c0 + j < D) {
          const int c = c0 + j;
          Vnew[r * D + c] = (float)nv[j];
          const T e = (T)w[c] - vh[j];
          res += (double)e * (double)e;
        }
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

// Q = sgn(M) for the d_F minimiser (one CTA).  Dynamic shared memory: 4 D x D doubles, 3 D x D floats.
__global__ void __launch_bounds__(256) polar_single_kernel(SpecScratch s, int D) {
  extern __shared__ __align__(16) double smp[];
  __shared__ double sh[32];
  const int DD = D * D;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) smp[e] = s.M[e];
  __syncthreads();
  float* f = reinterpret_cast<float*>(smp + 4 * DD);
  cta_polar_ns64(smp, smp + DD, smp + 2 * DD, smp + 3 * DD, f, f + DD, f + 2 * DD, D, sh);
  for (int e = threadIdx.x; e < DD; e += blockDim.x) s.Q[e] = smp[DD + e];
}

__global__ void __launch_bounds__(256) dist_generic_kernel(const float* __restrict__ X, const float* __restrict__ Yv,
                                                           long long rows, int D, SpecScratch s, Ctl* ctl) {
  extern __shared__ __align__(16) double smq[];
  __shared__ double sh[32];
  const int DD = D * D;
  for (int o = threadIdx.x; o < DD; o += blockDim.x) smq[o] = s.Q[o];
  __syncthreads();
  double acc = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < D; ++c) {
      double yq = 0.0;
      for (int k = 0; k < D; ++k) yq += (double)Yv[r * D + k] * smq[k * D + c];
      const double e = (double)X[r * D + c] - yq;
      acc += e * e;
    }
  }
  const double bs = block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(&s.scal[1], bs);
  if (last_block(&ctl->counter))
    if (threadIdx.x == 0) ctl->counter = 0u;
}

// ------------------------------------------------------------- launchers
int reduce_grid(long long rows);

static cudaError_t set_smem(const void* k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t generic_prepare(int d) {
  cudaError_t e;
  if ((e = set_smem((const void*)epilogue_generic_kernel, 5 * d * d * sizeof(float))) != cudaSuccess) return e;
  if ((e = set_smem((const void*)gpm_generic_kernel, 3 * d * d * sizeof(float))) != cudaSuccess) return e;
  const size_t polar_smem = 4 * d * d * sizeof(double) + 3 * d * d * sizeof(float);
  if ((e = set_smem((const void*)polar_generic_kernel, polar_smem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)polar_single_kernel, polar_smem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)update_generic_kernel<double>, 2 * d * d * sizeof(double))) != cudaSuccess) return e;
  if ((e = set_smem((const void*)update_generic_kernel<float>, 2 * d * d * sizeof(float))) != cudaSuccess) return e;
  if ((e = set_smem((const void*)gram_generic_kernel<float>, 2 * kRowsPerCta * ((d + 7) & ~7) * sizeof(float))) != cudaSuccess)
    return e;
  if ((e = set_smem((const void*)dist_generic_kernel, d * d * sizeof(double))) != cudaSuccess) return e;
  return set_smem((const void*)gram_generic_kernel<double>, 2 * kRowsPerCta * ((d + 7) & ~7) * sizeof(double));
}

static int gram_grid(long long rows) {
  long long g = (rows + kRowsPerCta - 1) / kRowsPerCta;
  return (int)(g < 256 ? (g < 1 ? 1 : g) : 256);
}

cudaError_t launch_epilogue_generic(const float* X, float* Y, float* Xout, int n, int d, float eta, int K,
                                    int safeguard, double tol, Ctl* ctl, double* upd_out, cudaStream_t st) {
  epilogue_generic_kernel<<<n, 256, 5 * d * d * sizeof(float), st>>>(X, Y, Xout, n, d, eta, K, safeguard, tol, ctl,
                                                                      upd_out);
  return cudaGetLastError();
}

cudaError_t launch_gpm_generic(const float* X, float* Y, float* Xout, int n, int d, double tol, Ctl* ctl,
                               cudaStream_t st) {
  gpm_generic_kernel<<<n, 256, 3 * d * d * sizeof(float), st>>>(X, Y, Xout, n, d, tol, ctl);
  return cudaGetLastError();
}

static cudaError_t launch_gram_finish(long long rows, int d, int mode, const SpecScratch& s, Ctl* ctl,
                                      cudaStream_t st) {
  const int nout = (mode == 0 ? 2 : 1) * d * d;
  gram_finish_kernel<<<(nout + 255) / 256, 256, d * d * sizeof(double), st>>>(gram_grid(rows), d, mode, s, ctl);
  return cudaGetLastError();
}

cudaError_t launch_spec_gram_generic(const float* V, float* Y, float* W, long long rows, int d, float shift,
                                     int dev_shift, int fp32, const SpecScratch& s, Ctl* ctl, cudaStream_t st) {
  if (fp32)
    gram_generic_kernel<float><<<gram_grid(rows), 256, 2 * kRowsPerCta * ((d + 7) & ~7) * sizeof(float), st>>>(
        V, Y, W, nullptr, rows, d, shift, dev_shift, 0, s, ctl);
  else
    gram_generic_kernel<double><<<gram_grid(rows), 256, 2 * kRowsPerCta * ((d + 7) & ~7) * sizeof(double), st>>>(
        V, Y, W, nullptr, rows, d, shift, dev_shift, 0, s, ctl);
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_gram_finish(rows, d, 0, s, ctl, st);
}

// count_pass == 2 (a pass of a rounded-operand product) runs the update in float32.
cudaError_t launch_spec_update_generic(const float* V, const float* W, float* Vnew, long long rows, int d,
                                       const SpecScratch& s, double tol, int count_pass, Ctl* ctl, cudaStream_t st) {
  if (count_pass == 2)
    update_generic_kernel<float><<<reduce_grid(rows), 256, 2 * d * d * sizeof(float), st>>>(V, W, Vnew, rows, d, s,
                                                                                          tol, count_pass, ctl);
  else
    update_generic_kernel<double><<<reduce_grid(rows), 256, 2 * d * d * sizeof(double), st>>>(V, W, Vnew, rows, d, s,
                                                                                            tol, count_pass, ctl);
  return cudaGetLastError();
}

cudaError_t launch_polar_generic(const float* V, float* X0, int n, int d, cudaStream_t st) {
  polar_generic_kernel<<<n, 256, 4 * d * d * sizeof(double) + 3 * d * d * sizeof(float), st>>>(V, X0, d);
  return cudaGetLastError();
}

cudaError_t launch_dF_generic(const float* X, const float* Yv, long long rows, int d, const SpecScratch& s, Ctl* ctl,
                              cudaStream_t st) {
  gram_generic_kernel<double><<<gram_grid(rows), 256, 2 * kRowsPerCta * ((d + 7) & ~7) * sizeof(double), st>>>(
      nullptr, const_cast<float*>(Yv), nullptr, X, rows, d, 0.f, 0, 1, s, ctl);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_gram_finish(rows, d, 1, s, ctl, st);
  if (e != cudaSuccess) return e;
  polar_single_kernel<<<1, 256, 4 * d * d * sizeof(double) + 3 * d * d * sizeof(float), st>>>(s, d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dist_generic_kernel<<<reduce_grid(rows), 256, d * d * sizeof(double), st>>>(X, Yv, rows, d, s, ctl);
  return cudaGetLastError();
}

}  // namespace nsrgs

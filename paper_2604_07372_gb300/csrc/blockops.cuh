// d x d per-block arithmetic shared by the single-instance and batched kernels:
// Algorithm 2's block update, the float64 matrix sign, Cholesky, and CTA-level
// float64 reductions.
#pragma once

#include <math.h>

#include "common.cuh"

namespace nsrgs {

// ------------------------------------------------------ float64 d x d polar
// One-sided Jacobi (Hestenes) SVD: rotate column pairs of U = M until they are
// orthogonal, accumulating the rotations in V; then U Sigma = M V and
// sgn(M) = (U Sigma) Sigma^{-1} V^T (§2.1's matrix sign, exact up to rounding).
template <int D>
__device__ inline void polar_fp64(const double (&M)[D][D], double (&Q)[D][D]) {
  double U[D][D], V[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      U[r][c] = M[r][c];
      V[r][c] = (r == c) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0;
#pragma unroll
    for (int p = 0; p < D - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < D; ++q) {
        double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          al += U[r][p] * U[r][p];
          be += U[r][q] * U[r][q];
          ga += U[r][p] * U[r][q];
        }
        const double nrm = sqrt(al * be);
        if (nrm == 0.0 || fabs(ga) <= 1e-17 * nrm) continue;
        off = fmax(off, fabs(ga) / nrm);
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = c * t;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          const double up = U[r][p], uq = U[r][q];
          U[r][p] = c * up - s * uq;
          U[r][q] = s * up + c * uq;
          const double vp = V[r][p], vq = V[r][q];
          V[r][p] = c * vp - s * vq;
          V[r][q] = s * vp + c * vq;
        }
      }
    if (off < 1e-15) break;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double s2 = 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) s2 += U[r][c] * U[r][c];
    const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) U[r][c] *= inv;
  }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) acc += U[r][k] * V[c][k];
      Q[r][c] = acc;
    }
}

// Same one-sided Jacobi in float32 (the GPU baseline of the generalised power
// method uses a float32 batched per-block SVD, like the float32 NS-RGS path).
template <int D>
__device__ inline void polar_fp32(const float (&M)[D][D], float (&Q)[D][D]) {
  float U[D][D], V[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      U[r][c] = M[r][c];
      V[r][c] = (r == c) ? 1.f : 0.f;
    }
  for (int sweep = 0; sweep < 20; ++sweep) {
    float off = 0.f;
#pragma unroll
    for (int p = 0; p < D - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < D; ++q) {
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          al = fmaf(U[r][p], U[r][p], al);
          be = fmaf(U[r][q], U[r][q], be);
          ga = fmaf(U[r][p], U[r][q], ga);
        }
        const float nrm = sqrtf(al * be);
        if (nrm == 0.f || fabsf(ga) <= 1e-8f * nrm) continue;
        off = fmaxf(off, fabsf(ga) / nrm);
        const float zeta = (be - al) / (2.f * ga);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float c = rsqrtf(1.f + t * t);
        const float s = c * t;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          const float up = U[r][p], uq = U[r][q];
          U[r][p] = c * up - s * uq;
          U[r][q] = s * up + c * uq;
          const float vp = V[r][p], vq = V[r][q];
          V[r][p] = c * vp - s * vq;
          V[r][q] = s * vp + c * vq;
        }
      }
    if (off < 1e-7f) break;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    float s2 = 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r) s2 = fmaf(U[r][c], U[r][c], s2);
    const float inv = s2 > 0.f ? rsqrtf(s2) : 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r) U[r][c] *= inv;
  }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(U[r][k], V[c][k], acc);
      Q[r][c] = acc;
    }
}

// ------------------------------------------------- block reductions (fp64)
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; result valid in thread 0.
__device__ inline double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Last-CTA election: returns true in every thread of the CTA that finishes last.
__device__ inline bool last_block(unsigned int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Cholesky G = R^T R (R upper) and R^{-1}, float64, one thread, D <= 64.
__device__ inline void chol_inv(const double* G, double* Rinv, int D, double* Rtmp) {
  for (int j = 0; j < D; ++j) {
    double s = G[j * D + j];
    for (int k = 0; k < j; ++k) s -= Rtmp[k * D + j] * Rtmp[k * D + j];
    const double rjj = sqrt(fmax(s, 1e-300));
    Rtmp[j * D + j] = rjj;
    for (int i = j + 1; i < D; ++i) {
      double t = G[j * D + i];
      for (int k = 0; k < j; ++k) t -= Rtmp[k * D + j] * Rtmp[k * D + i];
      Rtmp[j * D + i] = t / rjj;
    }
    for (int i = 0; i < j; ++i) Rtmp[j * D + i] = 0.0;
  }
  // upper-triangular inverse by back substitution, column by column
  for (int c = 0; c < D; ++c) {
    for (int r = D - 1; r >= 0; --r) {
      double t = (r == c) ? 1.0 : 0.0;
      for (int k = r + 1; k < D; ++k) t -= Rtmp[r * D + k] * Rinv[k * D + c];
      Rinv[r * D + c] = (r <= c) ? t / Rtmp[r * D + r] : 0.0;
    }
  }
}

// Is sym(H) - sigma I positive definite?  Cholesky with a relative pivot floor;
// one thread, M: D x D float64 scratch.
__device__ inline bool sym_shift_pd(const double* H, int D, double sigma, double floor_abs, double* M) {
  for (int j = 0; j < D; ++j) {
    double p = H[j * D + j] - sigma;
    for (int k = 0; k < j; ++k) p -= M[k * D + j] * M[k * D + j];
    if (!(p > floor_abs)) return false;
    const double rjj = sqrt(p);
    M[j * D + j] = rjj;
    for (int i = j + 1; i < D; ++i) {
      double t = 0.5 * (H[j * D + i] + H[i * D + j]);
      for (int k = 0; k < j; ++k) t -= M[k * D + j] * M[k * D + i];
      M[j * D + i] = t / rjj;
    }
  }
  return true;
}

// Spectral start, algebraic top-d test (Algorithm 2 asks for the eigenvectors of
// the d largest eigenvalues of A).  Subspace iteration on A_off + cI converges to
// the d eigenvalues of largest |lambda + c|.  At a converged basis V,
// H = V^T (A_off + cI) V holds the Ritz values theta_k + c.  When the symmetric
// part of H is positive definite, every eigenvalue left out has
// |lambda + c| <= min_k (theta_k + c), hence lambda <= min_k theta_k: the captured
// ones are the algebraic top d.  Otherwise a negative eigenvalue dominated and
// the start must run again with a shift that lifts the spectrum's negative end.
// The smallest eigenvalue mu of sym(H) (mu = min_k theta_k + c < 0) is bracketed
// by bisection between the Gershgorin lower bound and 0, each probe a Cholesky
// test (Sylvester's law of inertia), keeping the lower end lo <= mu; then
// c' = c - 5/4 lo + 1 > -min_k theta_k.
// Returns 0 when sym(H) is positive definite, else c'.  M: D x D float64
// scratch.  One thread; D <= 64.
__device__ inline double spec_shift_after(const double* H, int D, double c, double* M) {
  double dmax = 0.0;
  for (int k = 0; k < D; ++k) dmax = fmax(dmax, fabs(H[k * D + k]));
  const double floor_abs = 1e-12 * dmax;
  if (dmax > 0.0 && sym_shift_pd(H, D, 0.0, floor_abs, M)) return 0.0;
  double lo = 0.0;
  for (int k = 0; k < D; ++k) {
    double r = H[k * D + k];
    for (int l = 0; l < D; ++l)
      if (l != k) r -= 0.5 * fabs(H[k * D + l] + H[l * D + k]);
    lo = fmin(lo, r);
  }
  lo -= 1e-9 * dmax + 1e-300;  // strictly below the spectrum
  double hi = 0.0;
  for (int it = 0; it < 48 && hi - lo > 1e-6 * (fabs(lo) + 1.0); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sym_shift_pd(H, D, mid, 0.0, M)) lo = mid;
    else hi = mid;
  }
  return c - 1.25 * lo + 1.0;
}

// Entry e of the deterministic spectral start V^0 (any full-rank start works;
// entries uniform in (-1, 1), a splitmix64 hash of e).
__device__ __forceinline__ float spec_v0_entry(long long e) {
  unsigned long long z = (unsigned long long)e * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// End of a counted spectral pass (one thread): `tot` = ||W - V H||_F^2.  A restart
// pass only orthonormalises V^0.  Otherwise the relative residual is recorded
// and, once it is <= tol (or, with floor_max > 0, once it sits at the product's
// precision floor: at most floor_max and no smaller than the previous pass's),
// the algebraic top-d test decides: stop, or restart from V^0 with the larger
// shift (at most kSpecMaxRestarts times; after that the passes halt with
// spec_stop clear, reported as not converged).
__device__ inline void spec_finish_pass(double tot, int D, double tol, const SpecScratch& s, Ctl* ctl,
                                        double floor_max) {
  ctl->spec_iters += 1;
  if (ctl->spec_restart) {
    ctl->spec_restart = 0;
    return;
  }
  const double rel = sqrt(tot / fmax(s.scal[0], 1e-300));
  const double prev = ctl->spec_prev_res;
  ctl->spec_res = rel;
  ctl->spec_prev_res = rel;
  const bool at_floor = floor_max > 0.0 && prev > 0.0 && rel <= floor_max && rel >= prev;
  if (!(rel <= tol) && !at_floor) return;
  const double c2 = spec_shift_after(s.H, D, s.scal[3], s.M);
  if (c2 == 0.0) {
    ctl->spec_stop = 1;
    ctl->spec_skip = 1;
    if (!(rel <= tol)) ctl->flags |= FLAG_SPEC_AT_FLOOR;
  } else if (ctl->spec_round >= kSpecMaxRestarts) {
    ctl->spec_skip = 1;
  } else {
    s.scal[3] = c2;
    ctl->spec_restart = 1;
    ctl->spec_round += 1;
    ctl->spec_prev_res = 0.0;
    ctl->flags |= FLAG_SPEC_SHIFTED;
  }
}

// ---------------------------------------------------- Algorithm 2, one block
// For block i (Algorithm 2's loop body, §2.2 projection):
//   G = (n-1) X_i - Y_i,  P = (G - X_i G^T X_i)/2,  F = X_i - eta P,
//   S <- S (3I - S^T S)/2 applied K times (Algorithm 1), X_i^{t+1} = S.
// Y_i (= sum_{j != i} A_ij X_j) is zeroed for the next pass.  Adds
// ||X^{t+1}_i - X_i||^2 to diff2 and FLAG_* bits to flags.  With `safeguard`
// (beyond the paper) an F that fails Lemma 2.1's precondition, checked as
// ||I - F^T F||_F >= 1, starts the Newton-Schulz steps from F / ||F||_F (same
// polar factor, singular values in (0, 1]).
template <int D>
__device__ __forceinline__ void block_update(const float* __restrict__ X, float* __restrict__ Y,
                                             float* __restrict__ Xout, long long i, int n, float eta, int K,
                                             bool safeguard, double& diff2, unsigned int& flags) {
  float x[D][D], gm[D][D];
  const float nm1 = (float)(n - 1);
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const long long e = (i * D + r) * D + c;
      x[r][c] = X[e];
      gm[r][c] = nm1 * x[r][c] - Y[e];
      Y[e] = 0.f;
    }
  // T = G^T X
  float t[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(gm[k][r], x[k][c], acc);
      t[r][c] = acc;
    }
  // F = X - eta/2 (G - X T)
  float s[D][D];
  const float h = 0.5f * eta;
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float xt = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) xt = fmaf(x[r][k], t[k][c], xt);
      s[r][c] = x[r][c] - h * (gm[r][c] - xt);
    }
  // Lemma 2.1 precondition, checked with ||I - F^T F||_F (>= the spectral norm)
  {
    float e2 = 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float acc = (r == c) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) acc = fmaf(-s[k][r], s[k][c], acc);
        e2 = fmaf(acc, acc, e2);
      }
    if (!(e2 < 1.f)) {
      if (safeguard) {
        float f2 = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) f2 = fmaf(s[r][c], s[r][c], f2);
        const float inv = 1.f / sqrtf(f2);
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) s[r][c] *= inv;
        flags |= FLAG_NS_SAFEGUARDED;
      } else {
        flags |= FLAG_NS_PRECOND;
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    float m[D][D];  // 3I - S^T S
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float acc = (r == c) ? 3.f : 0.f;
#pragma unroll
        for (int l = 0; l < D; ++l) acc = fmaf(-s[l][r], s[l][c], acc);
        m[r][c] = acc;
      }
    float sn[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < D; ++l) acc = fmaf(s[r][l], m[l][c], acc);
        sn[r][c] = 0.5f * acc;
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) s[r][c] = sn[r][c];
  }
  bool finite = true;
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float v = s[r][c];
      finite = finite && isfinite(v);
      Xout[(i * D + r) * D + c] = v;
      const double dd = (double)v - (double)x[r][c];
      diff2 += dd * dd;
    }
  if (!finite) flags |= FLAG_NONFINITE;
}

}  // namespace nsrgs

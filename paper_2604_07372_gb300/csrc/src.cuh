// Element accessors of A_off for the packers: element (row, col) of the strict
// block-upper triangle (zero on and below the block diagonal and outside the
// matrix), read from the canonical upper-block list or from a dense matrix.
#pragma once

#include "common.cuh"

namespace nsrgs {

struct UpperSrc {
  const float* p;
  int n, d;
  __device__ float operator()(long long row, long long col) const {
    long long N = (long long)n * d;
    if (row >= N || col >= N) return 0.f;
    long long i = row / d, j = col / d;
    if (j <= i) return 0.f;
    long long a = row - i * d, bcol = col - j * d;
    long long idx = i * n - i * (i + 1) / 2 + (j - i - 1);
    return p[idx * d * d + a * d + bcol];
  }
};

struct DenseSrc {
  const float* p;
  int n, d;
  __device__ float operator()(long long row, long long col) const {
    long long N = (long long)n * d;
    if (row >= N || col >= N) return 0.f;
    if (col / d <= row / d) return 0.f;
    return p[row * N + col];
  }
};

// SE(d) form: element (row, col) of the strict block-upper triangle of the
// augmented matrix with (d+1) x (d+1) blocks
//     B_ij = [[A_ij, sqrt(kappa) c_ij], [0, w_ij]],   i < j,
// read from the upper-block lists of A (d x d) and c (d); w_ij = 1 when the
// pair is observed, i.e. A_ij has a nonzero entry (unobserved A_ij = 0).  With
// the iterate blocks [[X_j, 0], [sqrt(kappa) t_j^T, 1]] one symmetric product
// gives every pair sum of the SE(d) gradient.
struct SeAugSrc {
  const float* a;
  const float* c;
  int n, d;
  float sk;  // sqrt(kappa)
  __device__ float operator()(long long row, long long col) const {
    const int D = d + 1;
    const long long N = (long long)n * D;
    if (row >= N || col >= N) return 0.f;
    const long long i = row / D, j = col / D;
    if (j <= i) return 0.f;
    const int r = (int)(row - i * D), q = (int)(col - j * D);
    const long long idx = i * n - i * (i + 1) / 2 + (j - i - 1);
    if (r < d && q < d) return a[idx * d * d + r * d + q];
    if (r < d) return sk * c[idx * d + r];
    if (q < d) return 0.f;
    const float* blk = a + idx * d * d;
    for (int e = 0; e < d * d; ++e)
      if (blk[e] != 0.f) return 1.f;
    return 0.f;
  }
};

}  // namespace nsrgs

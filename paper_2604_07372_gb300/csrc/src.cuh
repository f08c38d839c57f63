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

}  // namespace nsrgs

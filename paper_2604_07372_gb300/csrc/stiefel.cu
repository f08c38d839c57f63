// Stiefel form (an extension the paper names, not part of its method): blocks
// X_i in R^{d x p}, p >= d, with orthonormal rows (X_i X_i^T = I_d), the
// Burer-Monteiro relaxation of O(d) synchronisation cited in §1.2.  Same
// objective (eq. (1)) and the same three steps as Algorithm 2:
//   Y = A_off X (nd x p),  C = X^T X (p x p, float64),
//   G_i = X_i (C - X_i^T X_i) - Y_i        (with X_j in O(d): (n-1) X_i - Y_i)
//   P_i = G_i - sym(G_i X_i^T) X_i          (tangent space: H X_i^T + X_i H^T = 0)
//   F_i = X_i - eta P_i,   S <- (3I - S S^T) S / 2, K times (Algorithm 1 by rows).
// With p = d every step is Algorithm 2's.  A is the dense float32 layout, or for
// d > 8 a symmetric tile layout (float32 or bfloat16 tiles, read once per
// product); the product's X has p columns.  The d x p work is one CTA per block
// in shared memory.
#include <math.h>
#include <string.h>

#include "blockops.cuh"

namespace nsrgs {

cudaError_t stream_dense_width(const void* packed, int n, int d, int width, const float* X, float* Y,
                               const int* skip, cudaStream_t st);
cudaError_t fs_sym_product_w(const void* packed, int n, int d, int width, const float* X, float* xt, float* Y,
                             Ctl* ctl, const int* skip, cudaStream_t st);
long long fs_sym_xt_bytes_w(int n, int d, int width);
bool fs_sym_supported(int d);
cudaError_t fs_sym_prepare(int d);
cudaError_t tc_sym_product_w(const void* packed, int n, int d, int width, const float* X, uint8_t* xt, float* Y,
                             Ctl* ctl, const int* skip, cudaStream_t st);
long long tc_sym_xt_bytes_w(int n, int d, int width);
bool tc_sym_width_ok(int d, int width);
cudaError_t tc_sym_prepare(int d, bool f8);
long long dense_pitch(int n, int d);
int reduce_grid(long long rows);

constexpr int kStGramThreads = 256;
constexpr int kStGramGrid = 128;

// C = X^T X over the nd rows of X (nd x p), float64, fixed-order sums: per-CTA
// partials, then the last CTA.  Thread t owns entries t, t + 256, ... of C.
__global__ void __launch_bounds__(kStGramThreads) stiefel_gram_kernel(const float* __restrict__ X, long long rows,
                                                                     int p, double* partials, double* C, Ctl* ctl) {
  if (ctl->stop) return;
  const int PP = p * p;
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
  const long long r0 = rows * blockIdx.x / gridDim.x, r1 = rows * (blockIdx.x + 1) / gridDim.x;
  for (long long r = r0; r < r1; ++r) {
    const float* x = X + r * p;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = threadIdx.x + j * kStGramThreads;
      if (e < PP) acc[j] += (double)x[e / p] * (double)x[e % p];
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = threadIdx.x + j * kStGramThreads;
    if (e < PP) partials[(size_t)blockIdx.x * PP + e] = acc[j];
  }
  if (!last_block(&ctl->counter)) return;
  for (int e = threadIdx.x; e < PP; e += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += partials[(size_t)b * PP + e];
    C[e] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->counter = 0u;
}

// One CTA per block i.  Shared memory (floats): x, g, s (d x p each), t (d x p),
// m (p x p), u (d x d).
__global__ void __launch_bounds__(256) stiefel_epilogue_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                                               const double* __restrict__ C, float* __restrict__ Xout,
                                                               int n, int d, int p, float eta, int K, double tol,
                                                               Ctl* ctl) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double sh[32];
  if (ctl->stop) return;
  const int DP = d * p, PP = p * p, DD = d * d;
  float* x = sm;
  float* g = x + DP;
  float* s = g + DP;
  float* t = s + DP;
  float* m = t + DP;
  float* u = m + PP;
  const long long base = (long long)blockIdx.x * DP;
  for (int e = threadIdx.x; e < DP; e += blockDim.x) x[e] = X[base + e];
  __syncthreads();
  // m = C - X_i^T X_i (float64 difference, then float32)
  for (int e = threadIdx.x; e < PP; e += blockDim.x) {
    const int a = e / p, b = e % p;
    double v = C[e];
    for (int k = 0; k < d; ++k) v -= (double)x[k * p + a] * (double)x[k * p + b];
    m[e] = (float)v;
  }
  __syncthreads();
  // g = x m - Y_i
  for (int e = threadIdx.x; e < DP; e += blockDim.x) {
    const int r = e / p, c = e % p;
    float v = 0.f;
    for (int a = 0; a < p; ++a) v = fmaf(x[r * p + a], m[a * p + c], v);
    g[e] = v - Y[base + e];
  }
  __syncthreads();
  // u = sym(g x^T)
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    const int r = e / d, q = e % d;
    float v1 = 0.f, v2 = 0.f;
    for (int c = 0; c < p; ++c) {
      v1 = fmaf(g[r * p + c], x[q * p + c], v1);
      v2 = fmaf(g[q * p + c], x[r * p + c], v2);
    }
    u[e] = 0.5f * (v1 + v2);
  }
  __syncthreads();
  // s = F = x - eta (g - u x)
  for (int e = threadIdx.x; e < DP; e += blockDim.x) {
    const int r = e / p, c = e % p;
    float ux = 0.f;
    for (int q = 0; q < d; ++q) ux = fmaf(u[r * d + q], x[q * p + c], ux);
    s[e] = x[e] - eta * (g[e] - ux);
  }
  __syncthreads();
  // Lemma 2.1 precondition for the row form: ||I - F F^T||_F < 1
  double e2 = 0.0;
  for (int e = threadIdx.x; e < DD; e += blockDim.x) {
    const int r = e / d, q = e % d;
    float v = 0.f;
    for (int c = 0; c < p; ++c) v = fmaf(s[r * p + c], s[q * p + c], v);
    const double w = (r == q ? 1.0 : 0.0) - (double)v;
    e2 += w * w;
  }
  e2 = block_sum(e2, sh);
  if (threadIdx.x == 0 && !(e2 < 1.0)) atomicOr(&ctl->flags, FLAG_NS_PRECOND);
  for (int k = 0; k < K; ++k) {
    __syncthreads();
    for (int e = threadIdx.x; e < DD; e += blockDim.x) {  // u = 3I - s s^T
      const int r = e / d, q = e % d;
      float v = 0.f;
      for (int c = 0; c < p; ++c) v = fmaf(s[r * p + c], s[q * p + c], v);
      u[e] = (r == q ? 3.f : 0.f) - v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < DP; e += blockDim.x) {  // t = u s / 2
      const int r = e / p, c = e % p;
      float v = 0.f;
      for (int q = 0; q < d; ++q) v = fmaf(u[r * d + q], s[q * p + c], v);
      t[e] = 0.5f * v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < DP; e += blockDim.x) s[e] = t[e];
  }
  __syncthreads();
  double diff2 = 0.0;
  bool finite = true;
  for (int e = threadIdx.x; e < DP; e += blockDim.x) {
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
      const double un = sqrt(tot / ((double)n * DP));
      ctl->last_upd = un;
      ctl->iters_done += 1;
      if (tol > 0.0 && un < tol) ctl->stop = 1;
      ctl->upd_acc = 0.0;
      ctl->counter = 0u;
    }
  }
}

__global__ void stiefel_copy_kernel(const float* __restrict__ X0, const float* __restrict__ X1, float* __restrict__ out,
                                    long long count, const Ctl* ctl) {
  const float* src = (ctl->iters_done & 1) ? X1 : X0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = src[e];
}

// ------------------------------------------------------------------ host
struct StiefelWs {
  Ctl* ctl;
  float* X[2];
  float* Y;
  double* C;
  double* partials;
  void* XT;  // d > 8: X^T tiles of the symmetric products
  size_t bytes;
};

static size_t st_align(size_t x) { return (x + 255) / 256 * 256; }

static StiefelWs map_stiefel(void* base, int n, int d, int p) {
  StiefelWs w{};
  size_t off = 0;
  uint8_t* b = reinterpret_cast<uint8_t*>(base);
  auto take = [&](size_t bytes) {
    uint8_t* q = b ? b + off : nullptr;
    off += st_align(bytes);
    return q;
  };
  const size_t vec = (size_t)n * d * p * sizeof(float) + 64 * p * sizeof(float);
  w.ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  w.X[0] = reinterpret_cast<float*>(take(vec));
  w.X[1] = reinterpret_cast<float*>(take(vec));
  w.Y = reinterpret_cast<float*>(take(vec));
  w.C = reinterpret_cast<double*>(take((size_t)p * p * sizeof(double)));
  w.partials = reinterpret_cast<double*>(take((size_t)kStGramGrid * p * p * sizeof(double)));
  if (d > 8) {
    const long long a = fs_sym_xt_bytes_w(n, d, p), c = tc_sym_xt_bytes_w(n, d, p);
    w.XT = take((size_t)(a > c ? a : c));
  }
  w.bytes = off;
  return w;
}

static size_t stiefel_smem(int d, int p) { return (size_t)(4 * d * p + p * p + d * d) * sizeof(float); }

}  // namespace nsrgs

using namespace nsrgs;

extern "C" size_t nsrgs_stiefel_workspace_bytes(int n, int d, int p) {
  if (n < 2 || d < 1 || p < d || p > 64) return 0;
  return map_stiefel(nullptr, n, d, p).bytes;
}

extern "C" nsrgs_status nsrgs_stiefel_solve(const nsrgs_A* A, int p, float eta, int T, int K, double tol,
                                            const float* X0, float* X, nsrgs_info* info, void* ws, size_t ws_bytes,
                                            void* stv) {
  NSRGS_CHECK_ARG(A && A->packed && X0 && X, "null argument");
  const int n = A->n, d = A->d;
  const bool sym_f32 = A->storage == NSRGS_F32 && d > 8 && fs_sym_supported(d);
  const bool sym_bf16 = A->storage == NSRGS_BF16 && d > 8 && d <= 64;
  NSRGS_CHECK_ARG(A->storage == NSRGS_DENSE_F32 || sym_f32 || sym_bf16,
                  "the Stiefel form streams NSRGS_DENSE_F32, or NSRGS_F32 / NSRGS_BF16 tiles for d > 8");
  NSRGS_CHECK_ARG(n >= 2 && d >= 1 && d <= 64 && (long long)n * d <= (1LL << 24), "n, d out of range");
  NSRGS_CHECK_ARG(p >= d && p <= 64, "need d <= p <= 64");
  NSRGS_CHECK_ARG(!sym_bf16 || tc_sym_width_ok(d, p),
                  "NSRGS_BF16 tiles need d and p in the same tile-width class (both <= 32 or both > 32)");
  NSRGS_CHECK_ARG(eta > 0.f && isfinite(eta), "eta must be finite and > 0");
  NSRGS_CHECK_ARG(T >= 0 && T <= 100000 && K >= 0 && K <= 64, "T in [0, 100000], K in [0, 64]");
  NSRGS_CHECK_ARG(tol >= 0.0 && isfinite(tol), "tol must be finite and >= 0");
  NSRGS_CHECK_ARG(ws && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0, "workspace must be 256-byte aligned");
  const StiefelWs need = map_stiefel(nullptr, n, d, p);
  if (ws_bytes < need.bytes) {
    set_error("workspace smaller than nsrgs_stiefel_workspace_bytes(n, d, p)");
    return NSRGS_ERR_NOMEM;
  }
  cudaStream_t st = (cudaStream_t)stv;
  const StiefelWs w = map_stiefel(ws, n, d, p);
  const size_t smem = stiefel_smem(d, p);
  NSRGS_CUDA_TRY(cudaFuncSetAttribute(stiefel_epilogue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (sym_f32) NSRGS_CUDA_TRY(fs_sym_prepare(p));
  if (sym_bf16) NSRGS_CUDA_TRY(tc_sym_prepare(p, false));
  const size_t ybytes = (size_t)n * d * p * sizeof(float) + 64 * p * sizeof(float);
  const long long count = (long long)n * d * p;
  NSRGS_CUDA_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(w.X[0], X0, count * sizeof(float), cudaMemcpyDeviceToDevice, st));
  for (int t = 0; t < T; ++t) {
    const float* Xt = w.X[t & 1];
    float* Xn = w.X[(t + 1) & 1];
    if (sym_f32 || sym_bf16) {  // the tile streams add into Y
      NSRGS_CUDA_TRY(cudaMemsetAsync(w.Y, 0, ybytes, st));
      if (sym_f32)
        NSRGS_CUDA_TRY(fs_sym_product_w(A->packed, n, d, p, Xt, reinterpret_cast<float*>(w.XT), w.Y, w.ctl,
                                        &w.ctl->stop, st));
      else
        NSRGS_CUDA_TRY(tc_sym_product_w(A->packed, n, d, p, Xt, reinterpret_cast<uint8_t*>(w.XT), w.Y, w.ctl,
                                        &w.ctl->stop, st));
    } else {
      NSRGS_CUDA_TRY(stream_dense_width(A->packed, n, d, p, Xt, w.Y, &w.ctl->stop, st));
    }
    stiefel_gram_kernel<<<kStGramGrid, kStGramThreads, 0, st>>>(Xt, (long long)n * d, p, w.partials, w.C, w.ctl);
    NSRGS_CUDA_TRY(cudaGetLastError());
    stiefel_epilogue_kernel<<<n, 256, smem, st>>>(Xt, w.Y, w.C, Xn, n, d, p, eta, K, tol, w.ctl);
    NSRGS_CUDA_TRY(cudaGetLastError());
  }
  stiefel_copy_kernel<<<reduce_grid(count), 256, 0, st>>>(w.X[0], w.X[1], X, count, w.ctl);
  NSRGS_CUDA_TRY(cudaGetLastError());
  if (info) {
    Ctl c{};
    NSRGS_CUDA_TRY(cudaMemcpyAsync(&c, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
    memset(info, 0, sizeof(*info));
    info->iters = c.iters_done;
    info->last_update_norm = c.last_upd;
    info->flags = c.flags & (FLAG_NONFINITE | FLAG_NS_PRECOND);
    info->objective = NAN;
    info->rel_decrease = NAN;
    if (c.flags & FLAG_NONFINITE) {
      set_error("an iterate became non-finite");
      return NSRGS_ERR_NONFINITE;
    }
  }
  return NSRGS_OK;
}

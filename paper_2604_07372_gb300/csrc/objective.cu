// The least-squares objective of eq. (1) and the relative decrease behind the
// stopping rule of §4.1, evaluated from the A-stream's product at no extra A
// traffic per iteration.
//
// With G = X^T X (d x d), s(X) = sum_i ||X_i^T X_i||_F^2 and Y = A_off X,
//   F(X) = 1/2 sum_{i != j} ||X_i X_j^T - A_ij||_F^2
//        = 1/2 (||G||_F^2 - s(X)) - tr(X^T Y) + 1/2 ||A_off||_F^2,
// because sum_{i != j} ||X_i X_j^T||^2 = ||G||^2 - s(X) and
// sum_{i != j} <X_i X_j^T, A_ij> = tr(X^T A_off X).
//
// The rule stops after the first iteration t with
//   R^t = (F(X^t) - F(X^{t+1})) / F(X^{t+1}) < rel_tol.
// F itself is a difference of terms up to ~n^2 d; in float32 the products Y
// carry rounding errors that would swamp a relative decrease of 1e-8.  So the
// decrease is evaluated in difference form: with D = X' - X (X' the newer
// iterate) and A_off symmetric,
//   tr(X'^T A X') - tr(X^T A X) = tr(D^T (A X + A X')),
// whose rounding error scales with ||D|| instead of ||X||, and the Gram terms
// come from float64 sums of exact float32 products:
//   F(X) - F(X') = 1/2 (<G - G', G + G'> - (s(X) - s(X'))) + tr(D^T (Y + Y')).
// All sums are taken in a fixed order (per-CTA partials, then the last CTA), so
// the stop decision is reproducible run to run.
#include <math.h>

#include "bcsr.cuh"
#include "blockops.cuh"
#include "tc_sym.cuh"

namespace nsrgs {

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

constexpr int kObjThreads = 256;
constexpr int kObjMaxGrid = 256;

// Blocks per CTA batch and Gram entries per thread.
__host__ __device__ inline int obj_nb(int D) { return D * D <= kObjThreads ? kObjThreads / (D * D) : 1; }
__host__ __device__ inline int obj_ept(int D) { return D * D <= kObjThreads ? 1 : (D * D + kObjThreads - 1) / kObjThreads; }

int obj_grid(int n, int D) {
  const int nb = obj_nb(D);
  long long g = ((long long)n + nb - 1) / nb;
  if (g > kObjMaxGrid) g = kObjMaxGrid;
  return (int)(g < 1 ? 1 : g);
}

// Per-CTA partials of an evaluation (d*d + 3 per CTA) or of the ||A_off||^2 pass (one per CTA).
size_t obj_partials_doubles(int n, int D) {
  const size_t a = (size_t)obj_grid(n, D) * (size_t)(D * D + 3);
  return a > (size_t)kObjMaxGrid ? a : (size_t)kObjMaxGrid;
}

// One evaluation at the current iterate Xc (with Yc = A_off Xc).  When the
// scratch holds a previous evaluation (scal[OBJ_HAVE_PREV] != 0), Xp / Yp are the
// previous iterate and its product, and R = (F(Xp) - F(Xc)) / F(Xc) is formed;
// R < rel_tol sets ctl->stop.  Yp receives Yc for the next evaluation.
__global__ void __launch_bounds__(kObjThreads) objective_kernel(const float* __restrict__ Xc,
                                                                const float* __restrict__ Yc,
                                                                const float* __restrict__ Xp, float* __restrict__ Yp,
                                                                int n, int D, double rel_tol, ObjScratch o, Ctl* ctl) {
  __shared__ double sh[32];
  __shared__ double gsh[kObjThreads];
  if (ctl->stop) return;
  const int DD = D * D;
  const int NB = obj_nb(D);
  const int EPT = obj_ept(D);
  const bool prev = o.scal[OBJ_HAVE_PREV] != 0.0;
  const int t = threadIdx.x;
  // entries owned by this thread: (slot, e0 + j*kObjThreads) for j < EPT
  const int slot = DD <= kObjThreads ? t / DD : 0;
  const int e0 = DD <= kObjThreads ? t % DD : t;
  const bool owner = DD <= kObjThreads ? slot < NB : true;

  double gacc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) gacc[j] = 0.0;
  double s = 0.0, tr = 0.0, trd = 0.0;
  for (long long b0 = (long long)blockIdx.x * NB; b0 < n; b0 += (long long)gridDim.x * NB) {
    const long long b = b0 + slot;
    if (!owner || b >= n) continue;
    const long long base = b * DD;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = e0 + j * kObjThreads;
      if (j < EPT && e < DD) {
        const int r = e / D, c = e % D;
        double g = 0.0;  // (X_b^T X_b)_{rc}
        for (int k = 0; k < D; ++k) g += (double)Xc[base + k * D + r] * (double)Xc[base + k * D + c];
        gacc[j] += g;
        s += g * g;
        const float x = Xc[base + e];
        const float y = Yc[base + e];
        tr += (double)x * (double)y;
        if (prev) trd += ((double)x - (double)Xp[base + e]) * ((double)Yp[base + e] + (double)y);
        Yp[base + e] = y;
      }
    }
  }

  // CTA partials: Gram entries (fixed-order sums over the batch slots), then s, tr, trd
  double* part = o.partials + (size_t)blockIdx.x * (DD + 3);
  if (DD <= kObjThreads) {
    gsh[t] = owner ? gacc[0] : 0.0;
    __syncthreads();
    if (t < DD) {
      double v = 0.0;
      for (int k = 0; k < NB; ++k) v += gsh[t + k * DD];
      part[t] = v;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = t + j * kObjThreads;
      if (j < EPT && e < DD) part[e] = gacc[j];
    }
  }
  const double bs = block_sum(s, sh);
  const double btr = block_sum(tr, sh);
  const double btrd = block_sum(trd, sh);
  if (t == 0) {
    part[DD] = bs;
    part[DD + 1] = btr;
    part[DD + 2] = btrd;
  }
  if (!last_block(&ctl->counter)) return;

  // last CTA: totals over the CTAs in order, then F and R
  const int P = DD + 3;
  double* tot = o.total;
  for (int e = t; e < P; e += kObjThreads) {
    double v = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) v += o.partials[(size_t)c * P + e];
    tot[e] = v;
  }
  __syncthreads();
  double gg = 0.0, dgg = 0.0;  // ||G||^2 and <Gp - G, Gp + G>
  for (int e = t; e < DD; e += kObjThreads) {
    const double g = tot[e];
    gg += g * g;
    if (prev) {
      const double gp = o.Gprev[e];
      dgg += (gp - g) * (gp + g);
    }
  }
  gg = block_sum(gg, sh);
  dgg = block_sum(dgg, sh);
  __syncthreads();
  if (t == 0) {
    const double sc = tot[DD], trc = tot[DD + 1], trdc = tot[DD + 2];
    const double F = 0.5 * (gg - sc) - trc + 0.5 * o.scal[OBJ_A2];
    double R = nan("");
    if (prev) {
      const double dF = 0.5 * (dgg - (o.scal[OBJ_S_PREV] - sc)) + trdc;
      R = F != 0.0 ? dF / F : 0.0;
      if (R < rel_tol) ctl->stop = 1;
    }
    o.scal[OBJ_F] = F;
    o.scal[OBJ_R] = R;
    o.scal[OBJ_S_PREV] = sc;
    o.scal[OBJ_HAVE_PREV] = 1.0;
    o.scal[OBJ_EVALS] += 1.0;
    ctl->counter = 0u;
  }
  for (int e = t; e < DD; e += kObjThreads) o.Gprev[e] = tot[e];
}

// ||A_off||_F^2 from the packed storage, partial sums per CTA in a fixed order.
// Flat arrays (dense layouts, FP32/BF16 panels): every stored value counts
// `weight` times (2 for the panels, which hold one triangle; zeros add nothing).
template <class T>
__global__ void __launch_bounds__(256) norm2_flat_kernel(const T* __restrict__ a, long long count, double weight,
                                                         ObjScratch o, Ctl* ctl) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = (double)to_float(a[e]);
    acc += v * v;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = acc;
  if (!last_block(&ctl->counter)) return;
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) v += o.partials[c];
    o.scal[OBJ_A2] = weight * v;
    ctl->counter = 0u;
  }
}

// Block-sparse rows (both triangles stored, each block once per direction):
// the stored values once.  The value array holds whole groups of 32 blocks; the
// padding of the last group is zero, so the sum runs over all its slots.
template <class T>
__global__ void __launch_bounds__(256) norm2_bcsr_kernel(const uint8_t* __restrict__ packed, int D, ObjScratch o,
                                                         Ctl* ctl) {
  __shared__ double sh[32];
  const long long* hdr = reinterpret_cast<const long long*>(packed);
  const long long count = bcsr_val_slots(hdr[2]) * D * D;
  const T* a = reinterpret_cast<const T*>(packed + hdr[4]);
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = (double)to_float(a[e]);
    acc += v * v;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = acc;
  if (!last_block(&ctl->counter)) return;
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) v += o.partials[c];
    o.scal[OBJ_A2] = v;
    ctl->counter = 0u;
  }
}

// FP8 panels: element (row, col) holds A/s_i with i = row / D, so each step's
// stored values are weighted by the square of their block row's scale.
__global__ void __launch_bounds__(256) norm2_fp8_panel_kernel(const uint8_t* __restrict__ packed, PanelGeom g,
                                                              ObjScratch o, Ctl* ctl) {
  __shared__ double sh[32];
  const long long* step_start = reinterpret_cast<const long long*>(packed + g.off_step_start);
  const long long* byte_off = reinterpret_cast<const long long*>(packed + g.off_byte_off);
  const float* scale = reinterpret_cast<const float*>(packed + g.off_scale);
  const uint8_t* panels = packed + g.header_bytes;
  double acc = 0.0;
  int b = 0;
  for (long long gs = blockIdx.x; gs < g.total_steps; gs += gridDim.x) {
    while (b + 1 < g.nslabs && step_start[b + 1] <= gs) ++b;  // steps visited in increasing order
    const long long q = gs - step_start[b];
    const int W = panel_warps(g, b, q);
    const uint8_t* src = panels + byte_off[b] + panel_step_offset(g, b, q);
    const long long elems = (long long)W * g.WB;  // one byte per element
    for (long long e = threadIdx.x; e < elems; e += blockDim.x) {
      // e -> (w, rt, lane, cc) in the order [w][rt][lane][cc]
      const int cc = (int)(e % g.CPT);
      long long t = e / g.CPT;
      const int lane = (int)(t % 32);
      t /= 32;
      const int rt = (int)(t % g.RT);
      const int w = (int)(t / g.RT);
      (void)cc;
      const long long row = (long long)b * g.RS + (long long)w * g.WROWS + (lane >> 2) * g.RT + rt;
      if (row >= (long long)g.n * g.D) continue;
      const float sc = scale[row / g.D];
      __half_raw h = __nv_cvt_fp8_to_halfraw(src[e], __NV_E4M3);
      const double v = (double)__half2float(*reinterpret_cast<__half*>(&h)) * sc;
      acc += v * v;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = acc;
  if (!last_block(&ctl->counter)) return;
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) v += o.partials[c];
    o.scal[OBJ_A2] = 2.0 * v;
    ctl->counter = 0u;
  }
}

// FP8 tile-upper layout: the stored triangle once, each E4M3 code times its
// block row's scale.  A CTA walks a contiguous range of the tile order.
template <int R>
__global__ void __launch_bounds__(256) norm2_ts8_kernel(const uint8_t* __restrict__ packed, int n, int d, ObjScratch o,
                                                       Ctl* ctl) {
  __shared__ double sh[32];
  __shared__ int tile_i;
  const int NT = ts_tile_rows(n, d);
  const long long rows = (long long)n * d;
  const float* scale = reinterpret_cast<const float*>(packed + ts8_scale_offset(n, d));
  const long long total = ts_tiles(NT);
  const long long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
  TsWalk<R> w;
  w.NT = NT;
  if (threadIdx.x == 0 && t0 < t1) w.seek(t0);
  double acc = 0.0;
  for (long long t = t0; t < t1; ++t) {
    __syncthreads();
    if (threadIdx.x == 0) {
      tile_i = w.I();
      bool se, ge;
      w.next(se, ge);
    }
    __syncthreads();
    const uint8_t* tile = packed + t * (long long)kTs8TileBytes;
    for (int e = threadIdx.x; e < kTs8TileBytes; e += blockDim.x) {
      const long long row = (long long)tile_i * kTsTile + ts8_row_of(e);
      if (row >= rows) continue;
      const __half_raw h = __nv_cvt_fp8_to_halfraw(tile[e], __NV_E4M3);
      const double v = (double)__half2float(__half(h)) * scale[row / d];
      acc += v * v;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = acc;
  if (!last_block(&ctl->counter)) return;
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) v += o.partials[c];
    o.scal[OBJ_A2] = 2.0 * v;
    ctl->counter = 0u;
  }
}

// ------------------------------------------------------------- launchers
cudaError_t launch_objective(const float* Xc, const float* Yc, const float* Xp, float* Yp, int n, int D,
                             double rel_tol, const ObjScratch& o, Ctl* ctl, cudaStream_t st) {
  objective_kernel<<<obj_grid(n, D), kObjThreads, 0, st>>>(Xc, Yc, Xp, Yp, n, D, rel_tol, o, ctl);
  return cudaGetLastError();
}

long long dense_pitch(int n, int d);
long long dense_bf16_pitch(int n, int d);
bool tc_sym_supported(int d);
long long tc_sym_bytes(int n, int d);
bool fs_sym_supported(int d);
long long fs_sym_bytes(int n, int d);

cudaError_t launch_norm2(const void* packed, int n, int d, int storage, const PanelGeom& g, const ObjScratch& o,
                         Ctl* ctl, cudaStream_t st) {
  const int grid = kObjMaxGrid;
  if (storage == NSRGS_DENSE_F32) {
    const long long count = (long long)n * d * dense_pitch(n, d);
    norm2_flat_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(packed), count, 1.0, o, ctl);
  } else if (storage == NSRGS_DENSE_BF16) {
    const long long count = (long long)n * d * dense_bf16_pitch(n, d);
    norm2_flat_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(packed), count, 1.0, o, ctl);
  } else if (storage == NSRGS_BCSR_F32) {
    norm2_bcsr_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const uint8_t*>(packed), d, o, ctl);
  } else if (storage == NSRGS_BCSR_BF16) {
    norm2_bcsr_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(reinterpret_cast<const uint8_t*>(packed), d, o, ctl);
  } else if (tile_storage(storage, d) && !tile_fp8(storage)) {
    // tile-upper layout: the upper triangle once, everything else zero
    norm2_flat_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(packed), tc_sym_bytes(n, d) / 2, 2.0,
                                            o, ctl);
  } else if (tile_storage(storage, d)) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(packed);
    const int w = ts_width(d);  // the visiting order follows the tile width
    if (w == 64) norm2_ts8_kernel<ts_strip_rows(64, true)><<<grid, 256, 0, st>>>(p, n, d, o, ctl);
    else if (w == 32) norm2_ts8_kernel<ts_strip_rows(32, true)><<<grid, 256, 0, st>>>(p, n, d, o, ctl);
    else norm2_ts8_kernel<ts_strip_rows(16, true)><<<grid, 256, 0, st>>>(p, n, d, o, ctl);
  } else if (storage == NSRGS_F32 && fs_sym_supported(d)) {
    // float32 tile-upper layout: the upper triangle once, everything else zero
    norm2_flat_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(packed), fs_sym_bytes(n, d) / 4, 2.0, o,
                                            ctl);
  } else if (storage == NSRGS_F32) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(packed) + g.header_bytes;
    norm2_flat_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(p), g.panel_bytes / 4, 2.0, o, ctl);
  } else if (storage == NSRGS_BF16) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(packed) + g.header_bytes;
    norm2_flat_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(p), g.panel_bytes / 2, 2.0, o,
                                            ctl);
  } else {
    norm2_fp8_panel_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const uint8_t*>(packed), g, o, ctl);
  }
  return cudaGetLastError();
}

}  // namespace nsrgs

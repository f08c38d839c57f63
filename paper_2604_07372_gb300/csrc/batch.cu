// Batched and served forms: many independent instances of different sizes
// advanced together.  One "tick" is
//   (1) one A-stream launch over every active instance's steps (the panel
//       kernel with a device table of instances, split evenly over the SMs),
//       each instance reading its own current X (spectral basis or iterate);
//   (2) one phase launch, one CTA per instance: a spectral pass (W = A V,
//       float64 Gram, Cholesky, V <- W R^{-1}, residual; on convergence the
//       exact blockwise sign gives X^0, Algorithm 2's start) or an NS-RGS
//       iteration (block_update for every block, update norm, stop test; on
//       stop X is copied to the caller's buffer).
// Instances therefore sit in different phases in the same tick.  A batch
// solve is an admit launch followed by (spectral passes + T) ticks replayed
// from a CUDA graph; the server (server.cu) runs ticks while it admits and
// retires requests between them.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "batch.cuh"
#include "bcsr.cuh"
#include "blockops.cuh"
#include "panel.cuh"

namespace nsrgs {

// ------------------------------------------------------------ the source
struct BatchSrc {
  const BatchDesc* descs;
  const long long* bases_;  // count + 1 entries: first global step of each instance
  int cnt;
  __device__ __forceinline__ int count() const { return cnt; }
  __device__ __forceinline__ int find(long long s) const { return find_first_leq(bases_, cnt, s); }
  __device__ __forceinline__ long long base(int i) const { return bases_[i]; }
  __device__ __forceinline__ InstView view(int i) const {
    const BatchDesc& d = descs[i];
    const Ctl* c = d.ctl;
    const int ph = c->phase;
    InstView v;
    v.packed = d.packed;
    v.Y = d.Y;
    v.ctl = d.ctl;
    v.g = d.g;
    if (ph == PHASE_SPEC) {
      v.X = d.X[(c->spec_iters + 1) & 1];
      v.skip = false;
    } else if (ph == PHASE_ITER) {
      v.X = d.X[c->iters_done & 1];
      v.skip = false;
    } else {
      v.X = d.X[0];
      v.skip = true;
    }
    return v;
  }
};

template <int D, int ST>
__global__ void __launch_bounds__(PCfg<D, ST>::THREADS, 1) panel_stream_batch_kernel(BatchSrc src) {
  panel_stream_body<D, ST>(src, src.base(src.cnt));
}

// ------------------------------------------------ per-instance kernels
// Prepares every instance in PHASE_ADMIT: clears its scratch, then either takes
// X^0 from the caller (start_given) or writes the start V^0 of the spectral
// subspace iteration, which the first (orthonormalising) pass turns into a basis.
template <int D>
__global__ void __launch_bounds__(256) batch_admit_kernel(const BatchDesc* descs, int* nspec) {
  const BatchDesc& d = descs[blockIdx.x];
  Ctl* c = d.ctl;
  if (c->phase != PHASE_ADMIT) return;
  const int n = d.g.n;
  const int rows = n * D;
  const long long vec = (long long)xpad_rows(n, D) * D;
  for (long long e = threadIdx.x; e < vec; e += blockDim.x) {
    d.Y[e] = 0.f;
    if (e >= (long long)rows * D) {
      d.X[0][e] = 0.f;
      d.X[1][e] = 0.f;
    }
  }
  __syncthreads();
  if (d.start_given) {
    for (long long e = threadIdx.x; e < (long long)rows * D; e += blockDim.x) d.X[0][e] = d.Xout[e];
  } else {
    for (long long e = threadIdx.x; e < (long long)rows * D; e += blockDim.x) d.X[0][e] = spec_v0_entry(e);
  }
  for (int e = threadIdx.x; e < kScrBytes / 8; e += blockDim.x) d.scr[e] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    d.scr[kScrShift] = 1.0;  // W = A_off V + V: subspace iteration on A itself
    c->spec_skip = 0;
    c->spec_restart = 0;
    c->spec_round = 0;
    c->spec_prev = 0;
    c->upd_acc = 0.0;
    c->last_upd = 0.0;
    c->spec_res = 0.0;
    c->counter = 0u;
    c->iters_done = 0;
    c->stop = 0;
    c->flags = 0u;
    c->spec_iters = 0;
    c->spec_stop = 0;
    c->phase = d.start_given ? (d.T > 0 ? PHASE_ITER : PHASE_DONE) : PHASE_SPEC0;
    if (!d.start_given) atomicAdd(nspec, 1);
  }
  if (d.start_given && d.T == 0) {
    // nothing to iterate: X^0 is the answer (already in the caller's buffer)
  }
}

// Instance of global block g for the CTA's chunk [g0, g0 + blockDim.x): thread 0
// bounds the chunk's instances once, each thread searches only that range.
// Call from every thread of the CTA.
__device__ __forceinline__ int chunk_instance(const long long* bbase, int cnt, long long g0, long long total,
                                              long long g, int* s_range) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long last = g0 + blockDim.x - 1 < total ? g0 + blockDim.x - 1 : total - 1;
    s_range[0] = find_first_leq(bbase, cnt, g0);
    s_range[1] = find_first_leq(bbase, cnt, last);
  }
  __syncthreads();
  if (g >= total) return -1;
  const int lo = s_range[0];
  return lo + find_first_leq(bbase + lo, s_range[1] - lo + 1, g);
}

// Segmented inclusive sum over runs of lanes that share a key (runs of an
// instance's consecutive blocks): on return the run's last lane holds the sum.
__device__ __forceinline__ double seg_sum(double v, int lane, int head) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= head) v += t;
  }
  return v;
}

// The spectral subspace pass over every instance in it, in two launches with a
// thread per block (bbase: first global block of each instance):
//  part 1: W = A V over the block's d rows (= Y + V; Y is zero in the first,
//          orthonormalising pass), Y cleared, and the float64 Gram partials
//          W^T W and V^T W summed per instance (segmented warp sums, atomics);
//          the lane that completes an instance forms R^{-1} from the Cholesky
//          of W^T W and keeps H = V^T W;
//  part 2: V_new = W R^{-1} and the residual ||W - V H||^2, summed per
//          instance; the completing lane takes the relative residual and the
//          stop decision (convergence or the pass cap moves the instance to
//          PHASE_POLAR, the orthonormalising pass to PHASE_SPEC).
// Basis buffers: pass s (spec_iters = s) reads V = X[(s + 1) & 1] and writes
// X[s & 1]; the orthonormalising pass reads X[0] and writes X[1], and so does a
// restart pass (PHASE_SPECR), whose V^0 is regenerated from its formula
// (spec_v0_entry) rather than read.
// Shift: passes iterate on A_off + cI (W = Y + cV), c = scr[kScrShift], starting
// at 1; when a pass converges, the algebraic top-d test (spec_shift_after)
// accepts the basis or moves the instance to PHASE_SPECR with a larger c.
template <int D>
__device__ __forceinline__ void spec_buffers(const BatchDesc& d, int ph, const float*& V, float*& Vn) {
  const int si = d.ctl->spec_iters;
  if (ph == PHASE_SPEC0 || ph == PHASE_SPECR) {
    V = d.X[0];
    Vn = d.X[1];
  } else {
    V = d.X[(si + 1) & 1];
    Vn = d.X[si & 1];
  }
}

template <int D>
__global__ void __launch_bounds__(256) batch_spec_gram_kernel(const BatchDesc* descs, const long long* bbase, int cnt,
                                                              const int* nspec) {
  constexpr int DD = D * D;
  __shared__ int s_range[2];
  if (*nspec == 0) return;  // no instance in a spectral pass (uniform)
  const int lane = threadIdx.x & 31;
  const long long total = bbase[cnt];
  for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < total; g0 += (long long)gridDim.x * blockDim.x) {
    const long long g = g0 + threadIdx.x;
    const int inst = chunk_instance(bbase, cnt, g0, total, g, s_range);
    const int ph = inst >= 0 ? descs[inst].ctl->phase : (int)PHASE_IDLE;
    const bool act = ph == PHASE_SPEC || ph == PHASE_SPEC0 || ph == PHASE_SPECR;
    double ww[DD], vw[DD];
#pragma unroll
    for (int o = 0; o < DD; ++o) ww[o] = vw[o] = 0.0;
    if (act) {
      const BatchDesc& d = descs[inst];
      const float* V;
      float* Vn;
      spec_buffers<D>(d, ph, V, Vn);
      const long long r0 = (g - bbase[inst]) * D;
      // the orthonormalising passes take W = V^0 (Y is zero there)
      const float shift = ph == PHASE_SPEC ? (float)d.scr[kScrShift] : 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        float v[D], w[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const long long e = (r0 + k) * D + c;
          v[c] = ph == PHASE_SPECR ? spec_v0_entry(e) : V[e];
          w[c] = ph == PHASE_SPEC ? d.Y[e] + shift * v[c] : v[c];
          d.W[e] = w[c];
          d.Y[e] = 0.f;
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            ww[a * D + b] += (double)w[a] * (double)w[b];
            vw[a * D + b] += (double)v[a] * (double)w[b];
          }
      }
    }
    const unsigned int m = __match_any_sync(0xffffffffu, act ? inst : -1);
    const int head = __ffs(m) - 1, tail = 31 - __clz(m);
#pragma unroll
    for (int o = 0; o < DD; ++o) {
      ww[o] = seg_sum(ww[o], lane, head);
      vw[o] = seg_sum(vw[o], lane, head);
    }
    if (act && lane == tail) {
      const BatchDesc& d = descs[inst];
      Ctl* c = d.ctl;
      double* scr = d.scr;
#pragma unroll
      for (int o = 0; o < DD; ++o) {
        atomicAdd(&scr[kScrWW + o], ww[o]);
        atomicAdd(&scr[kScrVW + o], vw[o]);
      }
      __threadfence();
      const unsigned int k = (unsigned int)__popc(m);
      if (atomicAdd(&c->counter, k) + k == (unsigned int)d.g.n) {
        __threadfence();
        double G[DD], R[DD], Rt[DD], h2 = 0.0;
#pragma unroll
        for (int o = 0; o < DD; ++o) {
          G[o] = atomicAdd(&scr[kScrWW + o], 0.0);
          const double h = atomicAdd(&scr[kScrVW + o], 0.0);
          scr[kScrH + o] = h;
          h2 += h * h;
          scr[kScrWW + o] = 0.0;
          scr[kScrVW + o] = 0.0;
        }
        chol_inv(G, R, D, Rt);
#pragma unroll
        for (int o = 0; o < DD; ++o) scr[kScrRinv + o] = R[o];
        scr[kScrH2] = h2;
        c->counter = 0u;
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(256) batch_spec_update_kernel(const BatchDesc* descs, const long long* bbase,
                                                                int cnt, int* nspec) {
  constexpr int DD = D * D;
  __shared__ int s_range[2];
  if (*nspec == 0) return;  // no instance in a spectral pass (uniform)
  const int lane = threadIdx.x & 31;
  const long long total = bbase[cnt];
  for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < total; g0 += (long long)gridDim.x * blockDim.x) {
    const long long g = g0 + threadIdx.x;
    const int inst = chunk_instance(bbase, cnt, g0, total, g, s_range);
    const int ph = inst >= 0 ? descs[inst].ctl->phase : (int)PHASE_IDLE;
    const bool act = ph == PHASE_SPEC || ph == PHASE_SPEC0 || ph == PHASE_SPECR;
    double res = 0.0;
    if (act) {
      const BatchDesc& d = descs[inst];
      const float* V;
      float* Vn;
      spec_buffers<D>(d, ph, V, Vn);
      double rinv[DD], hh[DD];
#pragma unroll
      for (int o = 0; o < DD; ++o) {
        rinv[o] = d.scr[kScrRinv + o];
        hh[o] = d.scr[kScrH + o];
      }
      const long long r0 = (g - bbase[inst]) * D;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        double v[D], w[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          v[c] = ph == PHASE_SPECR ? spec_v0_entry((r0 + k) * D + c) : V[(r0 + k) * D + c];
          w[c] = d.W[(r0 + k) * D + c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          double nv = 0.0, vh = 0.0;
#pragma unroll
          for (int q = 0; q < D; ++q) {
            nv += w[q] * rinv[q * D + c];
            vh += v[q] * hh[q * D + c];
          }
          Vn[(r0 + k) * D + c] = (float)nv;
          const double e = w[c] - vh;
          res += e * e;
        }
      }
    }
    const unsigned int m = __match_any_sync(0xffffffffu, act ? inst : -1);
    const int head = __ffs(m) - 1, tail = 31 - __clz(m);
    res = seg_sum(res, lane, head);
    if (act && lane == tail) {
      const BatchDesc& d = descs[inst];
      Ctl* c = d.ctl;
      atomicAdd(&d.scr[kScrRes], res);
      __threadfence();
      const unsigned int k = (unsigned int)__popc(m);
      if (atomicAdd(&c->counter, k) + k == (unsigned int)d.g.n) {
        __threadfence();
        const double tot = atomicAdd(&d.scr[kScrRes], 0.0);
        d.scr[kScrRes] = 0.0;
        if (ph == PHASE_SPEC0 || ph == PHASE_SPECR) {
          c->phase = PHASE_SPEC;
        } else {
          const int si = c->spec_iters;
          const double rel = sqrt(tot / fmax(d.scr[kScrH2], 1e-300));
          c->spec_res = rel;
          c->spec_iters = si + 1;
          bool done = c->spec_prev + si + 1 >= d.smax;  // the pass cap counts every round
          if (rel <= d.spec_tol) {
            // algebraic top-d test on H = V^T (A_off + cI) V of this pass
            double Hm[DD], tmp[DD];
#pragma unroll
            for (int o = 0; o < DD; ++o) Hm[o] = d.scr[kScrH + o];
            const double c2 = spec_shift_after(Hm, D, d.scr[kScrShift], tmp);
            if (c2 == 0.0) {
              c->spec_stop = 1;
              done = true;
            } else if (c->spec_round >= kSpecMaxRestarts) {
              done = true;  // spec_stop stays clear: reported as not converged
            } else if (!done) {
              d.scr[kScrShift] = c2;
              c->spec_round += 1;
              c->spec_prev += si + 1;
              c->spec_iters = 0;
              c->flags |= FLAG_SPEC_SHIFTED;
              c->phase = PHASE_SPECR;
            }
          }
          if (done) {
            c->phase = PHASE_POLAR;
            atomicSub(nspec, 1);
          }
        }
        c->counter = 0u;
      }
    }
  }
}

// The per-block part of a tick, thread per block over every instance's blocks
// (bbase: first global block of each instance, count + 1 entries), so that the
// largest instance's blocks are spread over the whole GPU:
//  PHASE_ITER:  Algorithm 2's update of block i (block_update), X^{t+1}_i also
//               written to the caller's X;
//  PHASE_POLAR: X^0_i = sgn(V_i), float64 polar (Algorithm 2's start).
// Lanes of a warp are grouped by instance (blocks are consecutive, so a group is
// a contiguous run of lanes); the group sums its update norms with a segmented
// scan and its last lane adds them and the group's block count to the
// instance's control block.  The lane whose count completes the instance
// finishes the iteration (update norm, stop test) or starts the iterations.
template <int D>
__global__ void __launch_bounds__(256) batch_block_kernel(const BatchDesc* descs, const long long* bbase, int cnt) {
  constexpr int DD = D * D;
  __shared__ int s_range[2];
  const int lane = threadIdx.x & 31;
  const long long total = bbase[cnt];
  for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < total; g0 += (long long)gridDim.x * blockDim.x) {
    const long long g = g0 + threadIdx.x;
    const int inst = chunk_instance(bbase, cnt, g0, total, g, s_range);
    const int ph = inst >= 0 ? descs[inst].ctl->phase : (int)PHASE_IDLE;
    const bool act = ph == PHASE_ITER || ph == PHASE_POLAR;
    double part = 0.0;
    if (act) {
      const BatchDesc& d = descs[inst];
      const long long i = g - bbase[inst];
      const long long base = i * DD;
      const int n = d.g.n;
      if (ph == PHASE_ITER) {
        const int it = d.ctl->iters_done;
        float* Xn = d.X[(it + 1) & 1];
        unsigned int flags = 0;
        block_update<D>(d.X[it & 1], d.Y, Xn, i, n, d.eta, d.K, d.safeguard != 0, part, flags);
        if (flags) atomicOr(&d.ctl->flags, flags);
#pragma unroll
        for (int e = 0; e < DD; ++e) d.Xout[base + e] = Xn[base + e];
      } else {
        const float* Vn = d.X[(d.ctl->spec_iters - 1) & 1];
        double M[D][D], Q[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) M[r][c] = Vn[base + r * D + c];
        polar_fp64<D>(M, Q);
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            d.X[0][base + r * D + c] = (float)Q[r][c];
            if (d.T == 0) d.Xout[base + r * D + c] = (float)Q[r][c];
          }
      }
    }
    const unsigned int m = __match_any_sync(0xffffffffu, act ? inst : -1);
    const int head = __ffs(m) - 1, tail = 31 - __clz(m);
    part = seg_sum(part, lane, head);
    if (act && lane == tail) {
      Ctl* c = descs[inst].ctl;
      const BatchDesc& d = descs[inst];
      if (ph == PHASE_ITER) atomicAdd(&c->upd_acc, part);
      __threadfence();
      const unsigned int k = (unsigned int)__popc(m);
      if (atomicAdd(&c->counter, k) + k == (unsigned int)d.g.n) {
        __threadfence();
        if (ph == PHASE_ITER) {
          const int it = c->iters_done;
          const double un = sqrt(atomicAdd(&c->upd_acc, 0.0) / ((double)d.g.n * D));
          c->last_upd = un;
          c->iters_done = it + 1;
          const bool conv = d.tol > 0.0 && un < d.tol;
          if (conv) c->stop = 1;
          if (it + 1 >= d.T || conv || (atomicOr(&c->flags, 0u) & FLAG_NONFINITE)) c->phase = PHASE_DONE;
        } else {
          c->iters_done = 0;
          c->phase = d.T > 0 ? PHASE_ITER : PHASE_DONE;
        }
        c->upd_acc = 0.0;
        c->counter = 0u;
      }
    }
  }
}

// Saves (to_w != 0) every instance's given start X^0 from the caller's buffer into
// its W scratch, or restores it from there: the autotuner runs two complete solves
// from the same start, and W is unused by solves that do not take the spectral start.
__global__ void batch_copy_start_kernel(const BatchDesc* descs, int to_w) {
  const BatchDesc& d = descs[blockIdx.x];
  const long long count = (long long)d.g.n * d.g.D * d.g.D;
  for (long long e = threadIdx.x; e < count; e += blockDim.x) {
    if (to_w) d.W[e] = d.Xout[e];
    else d.Xout[e] = d.W[e];
  }
}

// Compact per-instance report (one device-to-host copy for the whole batch).
__global__ void batch_report_kernel(const BatchDesc* descs, int count, BatchReport* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const Ctl* c = descs[i].ctl;
  BatchReport r;
  r.phase = c->phase;
  r.spec_iters = c->spec_prev + c->spec_iters;
  r.iters = c->iters_done;
  r.flags = c->flags;
  r.last_upd = c->last_upd;
  r.spec_res = c->spec_res;
  out[i] = r;
}

// Marks every instance of the table as admitted (start of a batch solve).
__global__ void batch_reset_kernel(const BatchDesc* descs, int count, int* nspec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *nspec = 0;
  if (i >= count) return;
  Ctl* c = descs[i].ctl;
  c->phase = PHASE_ADMIT;
  c->flags = 0u;
}

// ------------------------------------------------------------- launchers
// Block-sparse instances: one warp per global row; the row's instance by binary
// search over rbase (instances with no rows share their successor's base, and
// the last index with rbase <= r is the instance that owns row r).  Each
// instance reads its own current X as in the panel source.
template <int D, class T>
__global__ void __launch_bounds__(kBcsrWarps * 32) bcsr_batch_kernel(const BatchDesc* descs, const long long* rbase,
                                                                     int cnt) {
  __shared__ float xs[kBcsrWarps][BcsrX<D>::kSmemFloats];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long total = rbase[cnt];
  const long long nwarps = (long long)gridDim.x * kBcsrWarps;
  for (long long r = blockIdx.x * (long long)kBcsrWarps + w; r < total; r += nwarps) {
    const int inst = find_first_leq(rbase, cnt, r);
    const BatchDesc& d = descs[inst];
    const Ctl* c = d.ctl;
    const int ph = c->phase;
    const float* X;
    if (ph == PHASE_SPEC)
      X = d.X[(c->spec_iters + 1) & 1];
    else if (ph == PHASE_ITER)
      X = d.X[c->iters_done & 1];
    else
      continue;
    bcsr_row_product<D, T>(d.packed, r - rbase[inst], X, d.Y, lane, xs[w], d.ctl);
  }
}

cudaError_t batch_bcsr_stream(const BatchDesc* descs, const long long* rbase, int count, int d, int elem_bf16,
                              long long total_rows, cudaStream_t st) {
  // grid sized for the largest row total the table can hold; rows past the
  // current total return at once
  const long long g = std::max<long long>(
      1, std::min<long long>((total_rows + kBcsrWarps - 1) / kBcsrWarps, 32LL / kBcsrWarps * num_sms()));
#define L(DD)                                                                                             \
  if (elem_bf16)                                                                                          \
    bcsr_batch_kernel<DD, __nv_bfloat16><<<(unsigned)g, kBcsrWarps * 32, 0, st>>>(descs, rbase, count); \
  else                                                                                                    \
    bcsr_batch_kernel<DD, float><<<(unsigned)g, kBcsrWarps * 32, 0, st>>>(descs, rbase, count);
  switch (d) {
    case 1: L(1); break;
    case 2: L(2); break;
    case 3: L(3); break;
    case 4: L(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef L
  return cudaGetLastError();
}

template <int D, int ST>
static cudaError_t launch_batch_stream_t(const BatchSrc& s, cudaStream_t st, bool prepare) {
  using C = PCfg<D, ST>;
  if (prepare)
    return cudaFuncSetAttribute(panel_stream_batch_kernel<D, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                C::SMEM);
  panel_stream_batch_kernel<D, ST><<<num_sms(), C::THREADS, C::SMEM, st>>>(s);
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_batch_stream_d(const BatchSrc& s, int storage, cudaStream_t st, bool prepare) {
  switch (storage) {
    case NSRGS_F32: return launch_batch_stream_t<D, NSRGS_F32>(s, st, prepare);
    case NSRGS_BF16: return launch_batch_stream_t<D, NSRGS_BF16>(s, st, prepare);
    case NSRGS_FP8E4M3: return launch_batch_stream_t<D, NSRGS_FP8E4M3>(s, st, prepare);
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_stream(const BatchDesc* descs, const long long* base, int count, int d, int storage,
                         cudaStream_t st, bool prepare) {
  BatchSrc s{descs, base, count};
  switch (d) {
    case 1: return launch_batch_stream_d<1>(s, storage, st, prepare);
    case 2: return launch_batch_stream_d<2>(s, storage, st, prepare);
    case 3: return launch_batch_stream_d<3>(s, storage, st, prepare);
    case 4: return launch_batch_stream_d<4>(s, storage, st, prepare);
  }
  return cudaErrorInvalidValue;
}

#define NSRGS_BATCH_D(d, F)                \
  switch (d) {                             \
    case 1: F(1); break;                   \
    case 2: F(2); break;                   \
    case 3: F(3); break;                   \
    case 4: F(4); break;                   \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t batch_admit(const BatchDesc* descs, int count, int d, int* nspec, cudaStream_t st) {
#define L(DD) batch_admit_kernel<DD><<<count, 256, 0, st>>>(descs, nspec)
  NSRGS_BATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t batch_spec(const BatchDesc* descs, const long long* bbase, int count, int d, long long total_blocks,
                       int* nspec, cudaStream_t st) {
  const long long g = std::max<long long>(1, std::min<long long>((total_blocks + 255) / 256, 4LL * num_sms()));
#define L(DD)                                                                              \
  batch_spec_gram_kernel<DD><<<(unsigned)g, 256, 0, st>>>(descs, bbase, count, nspec);    \
  if (cudaPeekAtLastError() == cudaSuccess)                                                \
    batch_spec_update_kernel<DD><<<(unsigned)g, 256, 0, st>>>(descs, bbase, count, nspec);
  NSRGS_BATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t batch_block(const BatchDesc* descs, const long long* bbase, int count, int d, long long total_blocks,
                        cudaStream_t st) {
  const long long g = std::max<long long>(1, std::min<long long>((total_blocks + 255) / 256, 4LL * num_sms()));
#define L(DD) batch_block_kernel<DD><<<(unsigned)g, 256, 0, st>>>(descs, bbase, count)
  NSRGS_BATCH_D(d, L)
#undef L
  return cudaGetLastError();
}

cudaError_t batch_report(const BatchDesc* descs, int count, BatchReport* out, cudaStream_t st) {
  batch_report_kernel<<<(count + 127) / 128, 128, 0, st>>>(descs, count, out);
  return cudaGetLastError();
}

cudaError_t batch_reset(const BatchDesc* descs, int count, int* nspec, cudaStream_t st) {
  batch_reset_kernel<<<(count + 127) / 128, 128, 0, st>>>(descs, count, nspec);
  return cudaGetLastError();
}

// ------------------------------------------------------------ host layout
size_t batch_instance_bytes(int n, int d) {
  const size_t vec = ((size_t)xpad_rows(n, d) * d * sizeof(float) + 255) / 256 * 256;
  return 256 + kScrBytes + 4 * vec;
}

// Table region: descriptors | panel step bases | reports | block-sparse row bases |
// block bases | counters (256 bytes: instances in a spectral phase, the
// persistent form's work counter) | the persistent form's instance order.
size_t batch_table_bytes(int count) {
  const size_t t = ((size_t)count * sizeof(BatchDesc) + 255) / 256 * 256;
  const size_t b = ((size_t)(count + 1) * sizeof(long long) + 255) / 256 * 256;
  const size_t r = ((size_t)count * sizeof(BatchReport) + 255) / 256 * 256;
  const size_t o = ((size_t)count * sizeof(int) + 255) / 256 * 256;
  return t + 3 * b + r + 256 + o;
}

void fill_instance(BatchDesc& ds, uint8_t* region, int n, int d) {
  const size_t vec = ((size_t)xpad_rows(n, d) * d * sizeof(float) + 255) / 256 * 256;
  ds.ctl = reinterpret_cast<Ctl*>(region);
  ds.scr = reinterpret_cast<double*>(region + 256);
  uint8_t* v = region + 256 + kScrBytes;
  ds.X[0] = reinterpret_cast<float*>(v);
  ds.X[1] = reinterpret_cast<float*>(v + vec);
  ds.Y = reinterpret_cast<float*>(v + 2 * vec);
  ds.W = reinterpret_cast<float*>(v + 3 * vec);
}

}  // namespace nsrgs

using namespace nsrgs;

namespace {

struct BatchGraphKey {
  uint64_t hash;
  int count, d, storage, T, K, init, smax;
  double tol;
  void* ws;
  int dev;
  bool operator==(const BatchGraphKey& o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

std::mutex g_bmu;
std::vector<std::pair<BatchGraphKey, cudaGraphExec_t>> g_bgraphs;
cudaStream_t g_bcap[64] = {};
// Path of the batched form: requested (process-wide) and chosen per batch shape
// by timing both paths once (cached with the graph key).
int g_batch_path_req = NSRGS_BATCH_AUTO;
thread_local int g_batch_last_path = 0;
std::vector<std::pair<BatchGraphKey, int>> g_btuned;

uint64_t fnv(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

extern "C" size_t nsrgs_batch_workspace_bytes(const int* n, int count, int d) {
  if (!n || count < 1 || d < 1 || d > 4) return 0;
  size_t b = batch_table_bytes(count);
  for (int i = 0; i < count; ++i) {
    if (n[i] < 2) return 0;
    b += batch_instance_bytes(n[i], d);
  }
  return b;
}

extern "C" nsrgs_status nsrgs_batch_solve(const nsrgs_batch_item* items, int count, int d, int storage, int T, int K,
                                          double tol, int init, int spectral_max_iters, nsrgs_info* info, void* ws,
                                          size_t ws_bytes, void* stv) {
  NSRGS_CHECK_ARG(items != nullptr && count >= 1 && count <= (1 << 20), "items must be non-null, count >= 1");
  NSRGS_CHECK_ARG(d >= 1 && d <= 4, "the batched form covers 1 <= d <= 4");
  const bool sparse = storage == NSRGS_BCSR_F32 || storage == NSRGS_BCSR_BF16;
  NSRGS_CHECK_ARG((storage >= NSRGS_F32 && storage <= NSRGS_FP8E4M3) || sparse,
                  "batched storage must be F32, BF16, FP8E4M3, BCSR_F32 or BCSR_BF16");
  NSRGS_CHECK_ARG(T >= 0 && T <= 100000 && K >= 0 && K <= 64, "T in [0, 100000], K in [0, 64]");
  NSRGS_CHECK_ARG(tol >= 0.0 && isfinite(tol), "tol must be finite and >= 0");
  NSRGS_CHECK_ARG(!init || (spectral_max_iters >= 1 && spectral_max_iters <= 10000),
                  "spectral_max_iters must be in [1, 10000]");
  NSRGS_CHECK_ARG(ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0, "workspace must be 256-byte aligned");
  std::vector<int> ns(count);
  for (int i = 0; i < count; ++i) {
    const nsrgs_batch_item& it = items[i];
    NSRGS_CHECK_ARG(it.n >= 2 && (long long)it.n * d <= (1LL << 24), "every item needs n >= 2");
    NSRGS_CHECK_ARG(it.packed && (reinterpret_cast<uintptr_t>(it.packed) & 15u) == 0, "item packed must be 16-byte aligned");
    NSRGS_CHECK_ARG(it.X && (reinterpret_cast<uintptr_t>(it.X) & 15u) == 0, "item X must be 16-byte aligned");
    NSRGS_CHECK_ARG(it.eta > 0.f && isfinite(it.eta), "item eta must be finite and > 0");
    ns[i] = it.n;
  }
  const size_t need = nsrgs_batch_workspace_bytes(ns.data(), count, d);
  if (ws_bytes < need) {
    set_error("workspace smaller than nsrgs_batch_workspace_bytes");
    return NSRGS_ERR_NOMEM;
  }
  cudaStream_t st = (cudaStream_t)stv;
  // host image of the instance table
  uint8_t* base = reinterpret_cast<uint8_t*>(ws);
  const size_t tbytes = ((size_t)count * sizeof(BatchDesc) + 255) / 256 * 256;
  const size_t bbytes = ((size_t)(count + 1) * sizeof(long long) + 255) / 256 * 256;
  BatchDesc* d_descs = reinterpret_cast<BatchDesc*>(base);
  long long* d_base = reinterpret_cast<long long*>(base + tbytes);
  BatchReport* d_rep = reinterpret_cast<BatchReport*>(base + tbytes + bbytes);
  const size_t rbytes = ((size_t)count * sizeof(BatchReport) + 255) / 256 * 256;
  long long* d_rbase = reinterpret_cast<long long*>(base + tbytes + bbytes + rbytes);
  long long* d_bbase = reinterpret_cast<long long*>(base + tbytes + 2 * bbytes + rbytes);
  int* d_nspec = reinterpret_cast<int*>(base + tbytes + 3 * bbytes + rbytes);
  int* d_next = d_nspec + 1;
  int* d_order = reinterpret_cast<int*>(base + tbytes + 3 * bbytes + rbytes + 256);
  std::vector<BatchDesc> descs(count);
  std::vector<long long> bases(count + 1), rbases(count + 1), bbases(count + 1);
  size_t off = batch_table_bytes(count);
  long long steps = 0, rows = 0, blocks = 0;
  for (int i = 0; i < count; ++i) {
    BatchDesc& ds = descs[i];
    memset(&ds, 0, sizeof(ds));
    rbases[i] = rows;
    bbases[i] = blocks;
    blocks += items[i].n;
    if (sparse) {
      // no panel steps: the row kernel streams this instance
      ds.sparse = 1;
      ds.g.n = items[i].n;
      ds.g.D = d;
      ds.g.storage = storage;
      rows += items[i].n;
    } else if (!make_panel_geom(items[i].n, d, storage, &ds.g)) {
      set_error("unsupported (n, d, storage) in batch");
      return NSRGS_ERR_UNSUPPORTED;
    }
    ds.packed = reinterpret_cast<const uint8_t*>(items[i].packed);
    fill_instance(ds, base + off, items[i].n, d);
    off += batch_instance_bytes(items[i].n, d);
    ds.Xout = items[i].X;
    ds.eta = items[i].eta;
    ds.tol = tol;
    ds.spec_tol = 1e-6;
    ds.T = T;
    ds.K = K;
    ds.smax = init ? spectral_max_iters : 0;
    ds.start_given = init ? 0 : 1;
    ds.safeguard = items[i].ns_safeguard ? 1 : 0;
    ds.resident = sparse ? 0 : (persist_fits_resident(ds.g) ? 1 : 0);
    bases[i] = steps;
    steps += ds.g.total_steps;
  }
  bases[count] = steps;
  rbases[count] = rows;
  bbases[count] = blocks;
  // persistent form: instances in decreasing order of panel steps (the longest
  // solves start first, the short ones fill the tail)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return descs[a].g.total_steps > descs[b].g.total_steps; });
  if (!sparse) {
    NSRGS_CUDA_TRY(batch_stream(nullptr, nullptr, 0, d, storage, st, true));
    NSRGS_CUDA_TRY(batch_persist(nullptr, nullptr, 0, nullptr, d, storage, st, true));
  }
  NSRGS_CUDA_TRY(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(d_descs, descs.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(d_base, bases.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(d_rbase, rbases.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(d_bbase, bbases.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, st));

  int dev = 0;
  NSRGS_CUDA_TRY(cudaGetDevice(&dev));
  BatchGraphKey key;
  memset(&key, 0, sizeof(key));
  key.hash = fnv(descs.data(), sizeof(BatchDesc) * count);
  key.count = count;
  key.d = d;
  key.storage = storage;
  key.T = T;
  key.K = K;
  key.init = init ? 1 : 0;
  key.smax = init ? spectral_max_iters : 0;
  key.tol = tol;
  key.ws = ws;
  key.dev = dev;
  // ---- the tick path: admit + (passes + T) ticks replayed from a graph
  auto prepare_ticks = [&](cudaGraphExec_t* out) -> nsrgs_status {
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_bmu);
      for (auto& e : g_bgraphs)
        if (e.first == key) exec = e.second;
    }
    if (!exec) {
      if (!g_bcap[dev]) NSRGS_CUDA_TRY(cudaStreamCreateWithFlags(&g_bcap[dev], cudaStreamNonBlocking));
      cudaStream_t cs = g_bcap[dev];
      NSRGS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = batch_reset(d_descs, count, d_nspec, cs);
      if (e == cudaSuccess) e = batch_admit(d_descs, count, d, d_nspec, cs);
      // + the orthonormalising pass, + one orthonormalising pass per spectral restart
      const int ticks = (init ? spectral_max_iters + 1 + kSpecMaxRestarts : 0) + T;
      for (int t = 0; t < ticks && e == cudaSuccess; ++t) {
        e = sparse ? batch_bcsr_stream(d_descs, d_rbase, count, d, storage == NSRGS_BCSR_BF16, rows, cs)
                   : batch_stream(d_descs, d_base, count, d, storage, cs, false);
        if (e == cudaSuccess) e = batch_spec(d_descs, d_bbase, count, d, blocks, d_nspec, cs);
        if (e == cudaSuccess) e = batch_block(d_descs, d_bbase, count, d, blocks, cs);
      }
      if (e == cudaSuccess) e = batch_report(d_descs, count, d_rep, cs);
      cudaGraph_t graph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error(std::string("batch graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return NSRGS_ERR_CUDA;
      }
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        return NSRGS_ERR_CUDA;
      }
      std::lock_guard<std::mutex> lk(g_bmu);
      g_bgraphs.emplace_back(key, exec);
      if (g_bgraphs.size() > 8) {
        cudaGraphExecDestroy(g_bgraphs.front().second);
        g_bgraphs.erase(g_bgraphs.begin());
      }
    }
    *out = exec;
    return NSRGS_OK;
  };
  // ---- the persistent path: one launch over every instance, then the report
  auto launch_persist = [&]() -> nsrgs_status {
    NSRGS_CUDA_TRY(cudaMemsetAsync(d_next, 0, sizeof(int), st));
    NSRGS_CUDA_TRY(batch_persist(d_descs, d_order, count, d_next, d, storage, st, false));
    NSRGS_CUDA_TRY(batch_report(d_descs, count, d_rep, st));
    return NSRGS_OK;
  };
  int path = sparse ? NSRGS_BATCH_TICKS : g_batch_path_req;
  if (path == NSRGS_BATCH_AUTO) {
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto& e : g_btuned)
      if (e.first == key) path = e.second;
  }
  cudaGraphExec_t exec = nullptr;
  if (path == NSRGS_BATCH_AUTO) {
    // autotune: time both paths once on this batch (each run is a complete,
    // valid solve; the second one's results are the call's) and keep the faster
    nsrgs_status s2 = prepare_ticks(&exec);
    if (s2 != NSRGS_OK) return s2;
    cudaEvent_t ev[4];
    for (auto& e : ev) NSRGS_CUDA_TRY(cudaEventCreate(&e));
    if (!init) {  // both runs start from the caller's X^0: keep a copy for the second
      batch_copy_start_kernel<<<count, 256, 0, st>>>(d_descs, 1);
      NSRGS_CUDA_TRY(cudaGetLastError());
    }
    NSRGS_CUDA_TRY(cudaEventRecord(ev[0], st));
    NSRGS_CUDA_TRY(cudaGraphLaunch(exec, st));
    NSRGS_CUDA_TRY(cudaEventRecord(ev[1], st));
    if (!init) {
      batch_copy_start_kernel<<<count, 256, 0, st>>>(d_descs, 0);
      NSRGS_CUDA_TRY(cudaGetLastError());
    }
    NSRGS_CUDA_TRY(cudaEventRecord(ev[2], st));
    if ((s2 = launch_persist()) != NSRGS_OK) return s2;
    NSRGS_CUDA_TRY(cudaEventRecord(ev[3], st));
    NSRGS_CUDA_TRY(cudaEventSynchronize(ev[3]));
    float t_ticks = 0.f, t_persist = 0.f;
    NSRGS_CUDA_TRY(cudaEventElapsedTime(&t_ticks, ev[0], ev[1]));
    NSRGS_CUDA_TRY(cudaEventElapsedTime(&t_persist, ev[2], ev[3]));
    for (auto& e : ev) cudaEventDestroy(e);
    path = t_persist <= t_ticks ? NSRGS_BATCH_PERSISTENT : NSRGS_BATCH_TICKS;
    std::lock_guard<std::mutex> lk(g_bmu);
    g_btuned.emplace_back(key, path);
    if (g_btuned.size() > 64) g_btuned.erase(g_btuned.begin());
  } else if (path == NSRGS_BATCH_PERSISTENT) {
    nsrgs_status s2 = launch_persist();
    if (s2 != NSRGS_OK) return s2;
  } else {
    nsrgs_status s2 = prepare_ticks(&exec);
    if (s2 != NSRGS_OK) return s2;
    NSRGS_CUDA_TRY(cudaGraphLaunch(exec, st));
  }
  g_batch_last_path = path;
  if (info) {
    std::vector<BatchReport> rep(count);
    NSRGS_CUDA_TRY(cudaMemcpyAsync(rep.data(), d_rep, sizeof(BatchReport) * count, cudaMemcpyDeviceToHost, st));
    NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
    bool timeout = false, nonfinite = false, bad = false;
    for (int i = 0; i < count; ++i) {
      // an instance the persistent form did not finish (its CTA stopped on a flag)
      if (rep[i].phase != PHASE_DONE && path == NSRGS_BATCH_PERSISTENT) timeout = true;
      info[i].spectral_iters = rep[i].spec_iters;
      info[i].iters = rep[i].iters;
      info[i].last_update_norm = rep[i].last_upd;
      info[i].spectral_residual = rep[i].spec_res;
      info[i].objective = NAN;
      info[i].rel_decrease = NAN;
      info[i].flags = (rep[i].flags & (FLAG_NONFINITE | FLAG_NS_PRECOND | FLAG_NS_SAFEGUARDED | FLAG_SPEC_SHIFTED)) |
                      ((init && rep[i].spec_res > 1e-6) ? FLAG_SPEC_NOT_CONVERGED : 0u);
      timeout = timeout || (rep[i].flags & FLAG_TIMEOUT);
      bad = bad || (rep[i].flags & FLAG_BAD_LAYOUT);
      nonfinite = nonfinite || (rep[i].flags & FLAG_NONFINITE);
    }
    if (bad) {
      set_error("a packed A in the batch is inconsistent: an index or address left its buffer (access skipped)");
      return NSRGS_ERR_INVALID_ARG;
    }
    if (timeout) {
      set_error("a device-side wait timed out");
      return NSRGS_ERR_TIMEOUT;
    }
    if (nonfinite) {
      set_error("an iterate became non-finite in at least one instance");
      return NSRGS_ERR_NONFINITE;
    }
  }
  return NSRGS_OK;
}

extern "C" nsrgs_status nsrgs_batch_set_path(int path) {
  NSRGS_CHECK_ARG(path == NSRGS_BATCH_AUTO || path == NSRGS_BATCH_TICKS || path == NSRGS_BATCH_PERSISTENT,
                  "path must be NSRGS_BATCH_AUTO, NSRGS_BATCH_TICKS or NSRGS_BATCH_PERSISTENT");
  g_batch_path_req = path;
  return NSRGS_OK;
}

extern "C" int nsrgs_batch_last_path(void) { return g_batch_last_path; }

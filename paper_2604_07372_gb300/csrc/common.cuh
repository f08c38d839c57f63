// Internal definitions shared by the libnsrgs translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

#include "nsrgs.h"

namespace nsrgs {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
const char* get_error();

#define NSRGS_CUDA_TRY(expr)                                                      \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      ::nsrgs::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));     \
      return NSRGS_ERR_CUDA;                                                      \
    }                                                                             \
  } while (0)

#define NSRGS_CHECK_ARG(cond, msg)                                                \
  do {                                                                            \
    if (!(cond)) {                                                                \
      ::nsrgs::set_error(msg);                                                    \
      return NSRGS_ERR_INVALID_ARG;                                               \
    }                                                                             \
  } while (0)

// ------------------------------------------------------- device control
// One per workspace.  Written only by the library's kernels and by
// cudaMemsetAsync at the start of a call.
struct Ctl {
  double upd_acc;          // sum ||X^{t+1}_i - X^t_i||^2 of the running epilogue
  double last_upd;         // ||X^{t+1} - X^t||_F / sqrt(nd) of the last finished iteration
  double spec_res;         // spectral-init relative residual of the last pass
  double spec_res_acc;     // accumulator of the residual pass
  unsigned int counter;    // CTAs finished in the running epilogue / reduction
  int iters_done;          // NS-RGS iterations completed
  int stop;                // set when the update norm fell below tol
  unsigned int flags;      // FLAG_* bits
  int spec_iters;          // subspace iterations run
  int spec_stop;           // set when the subspace residual fell below tol
  int phase;               // batched / served instances: PHASE_*
  int spec_skip;           // spectral passes return at once (converged, or halted)
  int spec_restart;        // the next spectral pass restarts from V^0 with a larger shift
  int spec_round;          // restarts taken so far
  int spec_prev;           // batched / served instances: passes run before the last restart
  unsigned int gbar_count; // fused iteration loop: grid-barrier arrivals of the launch (monotonic)
  int pad;
  double upd_acc2[2];      // fused iteration loop: update-norm sums of even / odd iterations
  unsigned int ts8_max[2]; // FP8 tile-upper product: max |X| and max |s_i X_i| (float bits)
  double spec_prev_res;    // relative residual of the previous counted spectral pass (0: none since a start)
};

// A spectral start whose product rounds its operand (the tensor-core streams take
// V in bfloat16 or as E4M3 hi / lo planes) settles at a residual floor of about
// the operand's precision times ||A_off V_perp|| / ||A_off V||: below the floor
// further passes only move V within that rounding.  Such a start also stops once
// its residual, at most kSpecFloorMax, failed to decrease from one pass to the
// next (and reports FLAG_SPEC_AT_FLOOR).  The float32 tile stream (8 < d <= 64)
// sums thousands of float32 products per output; its floor sits near 1e-6 at
// n d = 64000..128000, so it stops the same way below kSpecFloorMaxF32.
constexpr double kSpecFloorMax = 1e-2;
constexpr double kSpecFloorMaxF32 = 1e-4;
// The counted-pass modes of the spectral update: 1 plain, 2 rounded-operand
// product (float32 d x d work, floor at kSpecFloorMax), 3 float32 tile stream
// (float64 d x d work, floor at kSpecFloorMaxF32).
__host__ __device__ constexpr double spec_floor_max(int count_pass) {
  return count_pass == 2 ? kSpecFloorMax : (count_pass == 3 ? kSpecFloorMaxF32 : 0.0);
}

// Storages held in the tile-upper tensor-core layout: BF16 and FP8E4M3 above d = 8
// (the CUDA-core panels at d <= 8; FP8 panels stop at d = 4).
__host__ __device__ inline bool tile_storage(int storage, int d) {
  return (storage == NSRGS_BF16 || storage == NSRGS_FP8E4M3) && d > 8 && d <= 64;
}
__host__ __device__ inline bool tile_fp8(int storage) { return storage == NSRGS_FP8E4M3; }

// Restarts the spectral start may take with a larger shift before it gives up
// (then it reports the subspace as not converged).
constexpr int kSpecMaxRestarts = 3;

// Phase of an instance in the batched and served forms.
enum : int {
  PHASE_IDLE = 0,   // slot unused
  PHASE_ADMIT = 1,  // admitted, start not prepared yet
  PHASE_SPEC = 2,   // spectral initialisation passes
  PHASE_ITER = 3,   // NS-RGS iterations
  PHASE_DONE = 4,   // finished; X copied to the caller
};

enum : unsigned int {
  FLAG_NONFINITE = 1u << 0,
  FLAG_NS_PRECOND = 1u << 1,
  FLAG_SPEC_NOT_CONVERGED = 1u << 2,
  FLAG_TIMEOUT = 1u << 3,
  FLAG_NS_SAFEGUARDED = 1u << 4,  // the safeguarded Newton-Schulz start was used for some block
  FLAG_BAD_LAYOUT = 1u << 5,      // a packed buffer's index or address left its buffer (access skipped)
  FLAG_SPEC_SHIFTED = 1u << 6,    // the spectral start restarted with a larger shift (see spec_shift_after)
  FLAG_SPEC_AT_FLOOR = 1u << 7,   // the spectral start stopped at its product's precision floor, above tol
};

// float64 scratch of the spectral initialisation and of d_F (all d x d unless noted).
struct SpecScratch {
  double* WW;        // W^T W
  double* H;         // V^T W
  double* Rinv;      // chol(W^T W)^{-1}
  double* M;         // scratch / Y^T X
  double* Q;         // sgn(Y^T X)
  double* scal;      // [0] ||H||_F^2, [1] d_F^2, [2] residual accumulator, [3] shift c of W = A_off V + c V
  double* partials;  // per-CTA partial sums
};

// float64 state of the objective evaluations (eq. (1), §4.1's stopping rule).
enum : int {
  OBJ_A2 = 0,         // ||A_off||_F^2 of the stored A
  OBJ_F = 1,          // F at the latest evaluated iterate
  OBJ_R = 2,          // relative decrease formed by the latest evaluation (NaN if none)
  OBJ_S_PREV = 3,     // sum_i ||X_i^T X_i||_F^2 at the latest evaluated iterate
  OBJ_HAVE_PREV = 4,  // nonzero once an evaluation has been stored
  OBJ_EVALS = 5,      // evaluations run
  OBJ_NSCAL = 8,
};
struct ObjScratch {
  double* scal;      // OBJ_* values
  double* Gprev;     // X^T X at the latest evaluated iterate (d x d)
  double* total;     // d*d + 3 totals of the running evaluation
  double* partials;  // per-CTA partial sums
  float* Yprev;      // A_off X at the latest evaluated iterate (n*d x d)
};

// ----------------------------------------------------------- panel geometry
// The symmetric read-once layout ("panel layout") of the packed strict
// block-upper triangle.  Block rows are grouped into slabs of SB block rows
// (RS = SB*D scalar rows).  Slab b starts at scalar column c0 = b*SB*D (its own
// diagonal block column) and runs to column n*D, cut into steps of SC columns.
// One step is the unit that one CTA stages in shared memory: up to NW warp
// slices of WB bytes each; warp slice w covers slab rows [w*WROWS, (w+1)*WROWS).
// Inside a warp slice the order is [row-in-thread rt][lane][LOADB bytes], lane =
// rg*4 + cg, so that the 32 lanes of a warp read 32 consecutive LOADB-byte
// vectors.  Steps that cross the slab's own diagonal square store only the
// warp slices that hold a nonzero block (a prefix, since rows below the
// staircase are zero); everything else in a stored slice that lies on or
// below the block diagonal, or past column n*D / row n*D, is stored as zero.
struct PanelGeom {
  int n, D, storage;
  int E;       // bytes per stored element
  int RT;      // scalar rows per thread
  int LOADB;   // bytes one thread loads per row and step
  int CPT;     // columns per thread (LOADB / E)
  int SC;      // columns per step (4*CPT)
  int NW;      // consumer warps per CTA
  int SB;      // block rows per slab (NW*8*RT / D)
  int RS;      // scalar rows per slab
  int WROWS;   // rows per warp slice (8*RT)
  int WB;      // bytes per warp slice (WROWS*SC*E)
  int nslabs;
  long long total_steps;
  long long panel_bytes;   // bytes of all stored warp slices
  long long header_bytes;  // bytes before the panels (tables, scales), 256-aligned
  // header layout (byte offsets from the packed base)
  long long off_step_start;  // int64[nslabs+1]: global index of each slab's first step
  long long off_byte_off;    // int64[nslabs+1]: byte offset of each slab's panels
  long long off_scale;       // float[n]: FP8 per-block-row scales (absent otherwise)
};

// Shape of the panel stream per (d, storage): scalar rows per thread (RT) and
// bytes loaded per row and step by one thread (LOADB).  A thread's d x d work is
// RT rows x LOADB/E columns against d X columns; RT and LOADB keep its row
// partials, X rows and column partials in registers (at most 168 with 10 warps
// per CTA, 146 with 14).  NW*8*RT (NW from panel_nw) must be a multiple of d so that slabs
// hold whole block rows.  Each step ends with a reduction of the CPT*d column partials over
// 8 lanes whose cost does not depend on RT, so a larger RT amortises it: at d = 4, RT = 8
// with 8 consumer warps ran 1.3x (FP32) to 1.7x (FP8) faster than RT = 4 with 12, and at
// d = 3 BF16 / FP8 (issue-bound) RT = 12 with 8 warps ran 10% / 8% faster than RT = 6 with 12;
// FP32 at d = 3 (bandwidth-bound) keeps RT = 6 with 12 warps; at d = 8, RT = 6 (three quarters
// of a block row per thread) ran 24% (FP32) / 28% (BF16) faster than RT = 4.
__host__ __device__ constexpr int panel_rt(int d, int storage) {
  return d <= 2 ? 8 : d == 3 ? (storage == NSRGS_F32 ? 6 : 12) : d == 4 ? 8 : d == 5 ? 5 : d == 6 ? 6 : d == 7 ? 7 : 6;
}
__host__ __device__ constexpr int panel_loadb(int d, int storage) {
  return storage == NSRGS_FP8E4M3 ? 8
         : d <= 4                 ? 16
         : d == 7                 ? (storage == NSRGS_F32 ? 8 : 4)
                                  : (storage == NSRGS_F32 ? 16 : 8);
}

// Consumer warps per CTA.  With the small tiles of d <= 2 and of FP32 at d = 3,
// 12 consumer warps (3 per scheduler) hide more of each step's latency
// (shared-memory loads, shuffles, barrier waits) and make each stage's bulk copy
// 1.5x larger: FP32 at d = 3 reaches the copy bandwidth with them (0.92 with 8).
// The larger per-thread tiles (BF16 / FP8 at d = 3, RT = 8 at d = 4, everything
// above) need the registers of 8 warps.
__host__ __device__ constexpr int panel_nw(int d, int storage) {
  return (d <= 2 || (d == 3 && storage == NSRGS_F32)) ? 12 : 8;
}

// Rows of X/Y padding needed by a layout (columns of the last step run past n*D).
__host__ __device__ inline int xpad_rows(int n, int D) { return n * D + 64; }

__host__ __device__ inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Number of warp slices stored for step q of slab b.
__host__ __device__ inline int panel_warps(const PanelGeom& g, int b, long long q) {
  long long c_end = (long long)b * g.SB * g.D + (q + 1) * g.SC;  // exclusive global column
  long long jmax = (c_end - 1) / g.D;                              // last block column touched
  if (jmax > g.n - 1) jmax = g.n - 1;
  long long rmax = (jmax - (long long)b * g.SB) * g.D;             // rows with a nonzero block
  long long rlim = ((long long)g.n - (long long)b * g.SB) * g.D;
  if (rmax > rlim) rmax = rlim;
  if (rmax > g.RS) rmax = g.RS;
  if (rmax < 1) rmax = 1;
  int w = (int)((rmax + g.WROWS - 1) / g.WROWS);
  return w < g.NW ? w : g.NW;
}

__host__ __device__ inline long long slab_steps(const PanelGeom& g, int b) {
  long long L = (long long)g.n * g.D - (long long)b * g.SB * g.D;
  return (L + g.SC - 1) / g.SC;
}

// Byte offset of step q inside slab b's panels.
__host__ __device__ inline long long panel_step_offset(const PanelGeom& g, int b, long long q) {
  long long off = 0;
  long long t = 0;
  for (; t < q; ++t) {
    int w = panel_warps(g, b, t);
    if (w == g.NW) break;
    off += (long long)w * g.WB;
  }
  off += (q - t) * (long long)g.NW * g.WB;
  return off;
}

bool make_panel_geom(int n, int d, int storage, PanelGeom* g);

// -------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: false after `limit_ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = globaltimer_ns();
  while (true) {
    for (int k = 0; k < 64; ++k)
      if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// 1-D bulk copy global -> shared through the TMA engine, completion on `bar`.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// L2 policy for data read once (the A stream): evicted first, so that it does not
// push out what is reused (X tiles, Y under its reduce-adds).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// bulk_g2s with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// (x0, x1) = (a0 b0 + c0, a1 b1 + c1): two float32 FMAs in one packed instruction,
// each rounded as fmaf rounds it (so results are those of the two fmaf calls).
__device__ __forceinline__ void fma2(float& x0, float& x1, float a0, float a1, float b0, float b1, float c0,
                                     float c1) {
  asm("{\n\t.reg .b64 a, b, c, d;\n\t"
      "mov.b64 a, {%2, %3};\n\t"
      "mov.b64 b, {%4, %5};\n\t"
      "mov.b64 c, {%6, %7};\n\t"
      "fma.rn.f32x2 d, a, b, c;\n\t"
      "mov.b64 {%0, %1}, d;\n\t}"
      : "=f"(x0), "=f"(x1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void red_add_v4_f32(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: far above any legitimate stage wait

// ------------------------------------------------------ launch helpers
int num_sms();
cudaError_t occupancy(const void* kernel, int threads, size_t smem, int* blocks_per_sm);

}  // namespace nsrgs

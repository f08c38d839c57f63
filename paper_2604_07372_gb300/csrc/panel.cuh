// The symmetric read-once A-stream (Y = A_off X), shared by the single-instance
// and the batched launches.
//
// Each stored block A_ij (i < j) of the strict block-upper triangle feeds both
// Y_i += A_ij X_j and Y_j += A_ij^T X_i (Algorithm 2's gradient needs
// sum_{j != i} A_ij X_j), so A is read once per iteration.
//
// Kernel structure (persistent, one CTA per SM, NW + 2 warps, NW from panel_nw):
//  * warp NW (producer): lane 0 walks the CTA's contiguous range of steps and
//    issues 1-D TMA bulk copies (cp.async.bulk) of each step's warp slices and
//    of the X rows of the step's columns into a ring of shared-memory stages,
//    completion tracked by mbarriers (expect_tx);
//  * warps 0..NW-1 (consumers): warp w owns slab rows [w*WROWS, (w+1)*WROWS);
//    lane (rg, cg) owns RT consecutive scalar rows and CPT consecutive columns
//    of each step.  Row partials of Y accumulate in registers across the whole walk
//    through a slab (reduced over the 4 cg lanes and added to Y once per slab).
//    Column partials of a step are reduced over the 8 rg lanes with shuffles
//    and written to a slot of a small shared-memory ring;
//  * warp NW+1 (reducer): sums a slot over the consumer warps and adds the
//    step's column partials to Y with red.global.add.v4.f32, then frees the
//    slot.  Consumers never wait for each other, only for data and slots.
// A "source" supplies the instances: one instance (from the kernel parameters)
// or a device table of instances whose steps are concatenated, so a batch of
// instances of different sizes is one evenly split launch.
// Every wait is bounded (globaltimer); a timeout sets FLAG_TIMEOUT in the
// instance's control block and ends the kernel instead of hanging.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace nsrgs {

template <int D, int ST>
struct PCfg {
  static constexpr int E = ST == NSRGS_F32 ? 4 : (ST == NSRGS_BF16 ? 2 : 1);
  static constexpr int RT = panel_rt(D, ST);
  static constexpr int LOADB = panel_loadb(D, ST);
  static constexpr int CPT = LOADB / E;
  static constexpr int SC = 4 * CPT;
  static constexpr int NW = panel_nw(D, ST);
  static constexpr int WROWS = 8 * RT;
  static constexpr int RS = NW * WROWS;
  static constexpr int SB = RS / D;
  static constexpr int WB = WROWS * SC * E;
  static constexpr int STAGE_A = NW * WB;
  static constexpr int STAGE_X = SC * D * 4;
  static constexpr int STAGE_BYTES = (STAGE_A + STAGE_X + 127) / 128 * 128;
  static constexpr int NSTAGE_RAW = (168 * 1024) / STAGE_BYTES;
  static constexpr int NSTAGE = NSTAGE_RAW > 12 ? 12 : (NSTAGE_RAW < 2 ? 2 : NSTAGE_RAW);
  static constexpr int NV = CPT * D;      // column-partial values per thread and step
  static constexpr int COLVALS = SC * D;  // column-partial values per warp and step
  static constexpr int RING = 4;          // column-partial slots between consumers and reducer
  static constexpr int THREADS = (NW + 2) * 32;
  // Column partials of a step are summed over the 8 row-group lanes by a shuffle
  // butterfly, or for FP8 storage through a per-warp shared-memory scratch
  // ([8][COLVALS + 4] floats, rows padded against bank conflicts): about half the
  // instructions, which pays where the kernel is most issue-bound (FP8: 5%
  // faster at d = 3; BF16 and FP32 measured level or slightly slower).
  static constexpr bool SMEM_RED = ST == NSRGS_FP8E4M3 && NV % 4 == 0;
  static constexpr int SCR_STRIDE = COLVALS + 4;
  static constexpr int SCR_FLOATS = SMEM_RED ? 8 * SCR_STRIDE : 0;
  // shared memory: stages | ring[RING][NW][COLVALS] | scratch[NW] |
  //                full[NSTAGE] empty[NSTAGE] cfull[RING] cempty[RING]
  static constexpr int OFF_RING = NSTAGE * STAGE_BYTES;
  static constexpr int OFF_SCR = OFF_RING + RING * NW * COLVALS * 4;
  static constexpr int OFF_BARS = OFF_SCR + NW * SCR_FLOATS * 4;
  static constexpr int SMEM = OFF_BARS + (2 * NSTAGE + 2 * RING) * 8;
  static_assert(COLVALS % 4 == 0 && COLVALS / 4 <= 32, "reducer lanes");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(RS % D == 0, "slabs of whole block rows");
};

// ---------------------------------------------------- column reduction
// Transposed butterfly over the 8 rg lanes (lane bits 4, 3, 2).  While the
// value count splits into whole columns the two partners exchange halves;
// otherwise they do a full exchange (and only one of them remains the owner).
template <int N, int D, int LVL>
struct RedLevel {
  static constexpr bool kSplit = (N % 2 == 0) && ((N / 2) % D == 0);
  static constexpr int kNext = kSplit ? N / 2 : N;
  static constexpr int kFinal = RedLevel<kNext, D, LVL + 1>::kFinal;
  __device__ __forceinline__ static void run(float* v, int lane, int& col0, bool& owner) {
    constexpr int mask = 16 >> LVL;
    const bool bit = (lane & mask) != 0;
    if constexpr (kSplit) {
      constexpr int H = N / 2;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        float send = bit ? v[k] : v[k + H];
        float keep = bit ? v[k + H] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
      }
      col0 += bit ? (H / D) : 0;
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], mask);
      owner = owner && !bit;
    }
    RedLevel<kNext, D, LVL + 1>::run(v, lane, col0, owner);
  }
};

template <int N, int D>
struct RedLevel<N, D, 3> {
  static constexpr int kFinal = N;
  __device__ __forceinline__ static void run(float*, int, int&, bool&) {}
};

// ---------------------------------------------------- element unpacking
// One thread's row load (LOADB bytes) as 32-bit words.
template <int LOADB>
struct RawVec;
template <>
struct RawVec<16> {
  using V = uint4;
  static constexpr int W = 4;
  __device__ __forceinline__ static void words(const V& x, uint32_t (&w)[W]) { w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w; }
};
template <>
struct RawVec<8> {
  using V = uint2;
  static constexpr int W = 2;
  __device__ __forceinline__ static void words(const V& x, uint32_t (&w)[W]) { w[0] = x.x; w[1] = x.y; }
};
template <>
struct RawVec<4> {
  using V = uint32_t;
  static constexpr int W = 1;
  __device__ __forceinline__ static void words(const V& x, uint32_t (&w)[W]) { w[0] = x; }
};
template <>
struct RawVec<2> {
  using V = uint16_t;
  static constexpr int W = 1;
  __device__ __forceinline__ static void words(const V& x, uint32_t (&w)[W]) { w[0] = x; }
};

// The CPT stored values of one thread's row load, widened to float32.
template <int ST, int CPT, int LOADB>
struct Unpack {
  using R = RawVec<LOADB>;
  using V = typename R::V;
  __device__ __forceinline__ static void run(const V& x, float (&o)[CPT]) {
    uint32_t w[R::W];
    R::words(x, w);
    if constexpr (ST == NSRGS_F32) {
#pragma unroll
      for (int k = 0; k < CPT; ++k) o[k] = __uint_as_float(w[k]);
    } else if constexpr (ST == NSRGS_BF16) {
#pragma unroll
      for (int k = 0; k < CPT / 2; ++k) {
        o[2 * k] = __uint_as_float(w[k] << 16);
        o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPT / 2; ++k) {
        const uint32_t pair = (w[k / 2] >> (16 * (k & 1))) & 0xffffu;
        __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<__half2*>(&h));
        o[2 * k] = a.x;
        o[2 * k + 1] = a.y;
      }
    }
  }
};

__device__ __forceinline__ int find_first_leq(const long long* starts, int count, long long s) {
  int lo = 0, hi = count - 1;  // last index with starts[idx] <= s
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One instance as the kernel sees it.
struct InstView {
  const uint8_t* packed;
  const float* X;  // padded, n*D + 64 rows
  float* Y;        // padded accumulator, zero on entry
  Ctl* ctl;
  PanelGeom g;
  bool skip;
};

// Position in the walk over one instance's steps, in 32-bit arithmetic with
// the geometry's compile-time constants.  W (stored warp slices of the step)
// is nondecreasing along a slab, so it is recomputed only until it reaches NW.
template <class C, int D>
struct Walk {
  const long long* step_start;
  int nslabs, n;
  int b, q, Sb, W;
  bool ragged;

  __device__ __forceinline__ int warps() const {
    const int c_end = b * C::SB * D + (q + 1) * C::SC;
    int jmax = (c_end - 1) / D;
    jmax = jmax < n - 1 ? jmax : n - 1;
    int rmax = (jmax - b * C::SB) * D;
    const int rlim = (n - b * C::SB) * D;
    rmax = rmax < rlim ? rmax : rlim;
    rmax = rmax < C::RS ? rmax : C::RS;
    rmax = rmax > 1 ? rmax : 1;
    const int w = (rmax + C::WROWS - 1) / C::WROWS;
    return w < C::NW ? w : C::NW;
  }
  __device__ __forceinline__ void refresh() {
    if (ragged) {
      W = warps();
      ragged = W < C::NW;
    }
  }
  __device__ __forceinline__ void start(const InstView& v, long long local_step) {
    step_start = reinterpret_cast<const long long*>(v.packed + v.g.off_step_start);
    nslabs = v.g.nslabs;
    n = v.g.n;
    b = find_first_leq(step_start, nslabs, local_step);
    q = (int)(local_step - step_start[b]);
    Sb = (int)(step_start[b + 1] - step_start[b]);
    ragged = true;
    refresh();
  }
  // Returns true when the walk left slab b (the caller flushes it).
  __device__ __forceinline__ bool advance() {
    if (++q < Sb) {
      refresh();
      return false;
    }
    ++b;
    q = 0;
    if (b < nslabs) {
      Sb = (int)(step_start[b + 1] - step_start[b]);
      ragged = true;
      refresh();
    }
    return true;
  }
  __device__ __forceinline__ int xcol() const { return b * C::SB * D + q * C::SC; }
};

// Runs `fn(view, lo, hi)` for every instance segment [lo, hi) (local step
// indices) of the global step range [g0, g1), in order.
template <class Src, class Fn>
__device__ __forceinline__ void for_segments(const Src& src, long long g0, long long g1, Fn&& fn) {
  int inst = src.find(g0);
  long long s = g0;
  while (s < g1 && inst < src.count()) {
    const long long base = src.base(inst);
    const long long end = src.base(inst + 1);
    const long long hi = end < g1 ? end : g1;
    if (hi > s) {
      const InstView v = src.view(inst);
      if (!fn(v, s - base, hi - base)) return;
    }
    s = hi;
    ++inst;
  }
}

// Pipeline position of one thread across calls of panel_stream_range: stage and
// ring indices with their mbarrier phases and the running step count, so a
// persistent kernel can stream the same CTA through many passes without
// re-initialising its barriers.
struct PanelPipe {
  int st = 0;        // stage ring index (producer, consumers)
  uint32_t ph = 0;   // its phase
  int slot = 0;      // column-partial ring index (consumers, reducer)
  uint32_t cph = 0;  // its phase
  long long it = 0;  // steps issued (producer) / consumed (consumers) so far
};

// Residency modes of panel_stream_range.  RES_RING streams every step through
// the ring of stages.  A CTA that owns a whole small instance can keep it in
// shared memory: RES_LOAD copies every step's stored warp slices and X rows to
// its own place in a dense area (step s at the sum of the earlier steps'
// W*WB + STAGE_X bytes, no stage reused), RES_KEEP copies only the X rows
// there and reads the warp slices left by the RES_LOAD pass.
enum : int { RES_RING = 0, RES_LOAD = 1, RES_KEEP = 2 };

// Initialises the stage and ring barriers (thread 0; the caller synchronises).
template <int D, int ST>
__device__ __forceinline__ void panel_init_barriers() {
  using C = PCfg<D, ST>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::OFF_BARS);
  uint64_t* empty = full + C::NSTAGE;
  uint64_t* cfull = empty + C::NSTAGE;
  uint64_t* cempty = cfull + C::RING;
  for (int s = 0; s < C::NSTAGE; ++s) {
    mbar_init(&full[s], 1);
    mbar_init(&empty[s], C::NW);
  }
  for (int s = 0; s < C::RING; ++s) {
    mbar_init(&cfull[s], C::NW);
    mbar_init(&cempty[s], 1);
  }
  fence_mbar_init();
}

// Streams the global step range [g0, g1) of `src` through this CTA.  Every
// thread of the CTA calls it; warps leave it at different times (the caller
// synchronises afterwards when it needs the result).  Barriers must have been
// initialised; `pp` carries the thread's pipeline position between calls.
// Sources whose panels are read once per pass (one instance streamed from HBM)
// declare kStreamOnce = true: their copies carry an L2 evict-first policy so that
// they do not push X and Y out of L2.  The batched sources keep the default
// policy, under which small instances stay in L2 from one pass to the next.
template <class S, class = void>
struct stream_once : std::false_type {};
template <class S>
struct stream_once<S, std::void_t<decltype(S::kStreamOnce)>> : std::bool_constant<S::kStreamOnce> {};

template <int D, int ST, class Src>
__device__ __forceinline__ void panel_stream_range(const Src& src, long long g0, long long g1, PanelPipe& pp,
                                                   int res_mode) {
  using C = PCfg<D, ST>;
  extern __shared__ __align__(128) uint8_t smem[];
  float* ring = reinterpret_cast<float*>(smem + C::OFF_RING);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::OFF_BARS);
  uint64_t* empty = full + C::NSTAGE;
  uint64_t* cfull = empty + C::NSTAGE;
  uint64_t* cempty = cfull + C::RING;
  const bool resident = res_mode != RES_RING;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (warp == C::NW) {
    // ------------------------------------------------------------- producer
    if (lane == 0) {
    // X may have been written by generic stores since the last pass (of this
    // launch, in a persistent kernel): order them before this thread's bulk copies
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const uint64_t pol = l2_evict_first_policy();
    int& st = pp.st;
    uint32_t& ph = pp.ph;
    long long& issued = pp.it;
    const long long issued0 = issued;
    uint32_t roff = 0;  // resident modes: dense offset of the current step
    bool ok = true;
    for_segments(src, g0, g1, [&](const InstView& v, long long lo, long long hi) {
      if (v.skip) return true;
      Walk<C, D> wk;
      wk.start(v, lo);
      const long long* byte_off = reinterpret_cast<const long long*>(v.packed + v.g.off_byte_off);
      const uint8_t* panels = v.packed + v.g.header_bytes;
      long long off = byte_off[wk.b] + panel_step_offset(v.g, wk.b, wk.q);
      for (long long s = lo; s < hi; ++s) {
        if (issued >= C::NSTAGE && !mbar_wait_bounded(&empty[st], ph ^ 1u, kWaitLimitNs)) {
          atomicOr(&v.ctl->flags, FLAG_TIMEOUT);
          ok = false;
          return false;
        }
        const uint32_t bytesA = (uint32_t)wk.W * C::WB;
        const uint8_t* srcA = panels + off;
        const float* srcX = v.X + (long long)wk.xcol() * D;
        // a copy that would leave the panels (either end: the offsets come from
        // the packed header) or start off a 16-byte boundary is refused and
        // flagged (the consumers then time out and return)
        if (off < 0 || off + bytesA > v.g.panel_bytes ||
            ((reinterpret_cast<uintptr_t>(srcA) | reinterpret_cast<uintptr_t>(srcX)) & 15u)) {
          atomicOr(&v.ctl->flags, FLAG_BAD_LAYOUT);
          ok = false;
          return false;
        }
        if (resident) {
          // each step keeps its own place: A slices, then the step's X rows; the
          // dense area is the stage ring's space
          if (roff + bytesA + C::STAGE_X > (uint32_t)C::OFF_RING) {
            atomicOr(&v.ctl->flags, FLAG_BAD_LAYOUT);
            ok = false;
            return false;
          }
          uint8_t* dst = smem + roff;
          if (res_mode == RES_LOAD) {
            mbar_arrive_expect_tx(&full[st], bytesA + C::STAGE_X);
            bulk_g2s(dst, srcA, bytesA, &full[st]);
          } else {
            mbar_arrive_expect_tx(&full[st], C::STAGE_X);
          }
          bulk_g2s(dst + bytesA, srcX, C::STAGE_X, &full[st]);
          roff += bytesA + C::STAGE_X;
        } else {
          uint8_t* stage = smem + st * C::STAGE_BYTES;
          mbar_arrive_expect_tx(&full[st], bytesA + C::STAGE_X);
          if constexpr (stream_once<Src>::value)
            bulk_g2s_hint(stage, srcA, bytesA, &full[st], pol);
          else
            bulk_g2s(stage, srcA, bytesA, &full[st]);
          bulk_g2s(stage + C::STAGE_A, srcX, C::STAGE_X, &full[st]);
        }
        off += bytesA;
        if (wk.advance() && wk.b < wk.nslabs) off = byte_off[wk.b];
        ++issued;
        if (++st == C::NSTAGE) {
          st = 0;
          ph ^= 1u;
        }
      }
      return true;
    });
    (void)ok;
    // Do not leave while copies into this CTA's shared memory may be in flight.
    const long long first = issued - C::NSTAGE > issued0 ? issued - C::NSTAGE : issued0;
    for (long long k = first; k < issued; ++k)
      if (!mbar_wait_bounded(&full[k % C::NSTAGE], (uint32_t)((k / C::NSTAGE) & 1), kWaitLimitNs)) break;
    }
    __syncwarp();
    return;
  }

  if (warp == C::NW + 1) {
    // -------------------------------------------------------------- reducer
    int& slot = pp.slot;
    uint32_t& ph = pp.cph;
    for_segments(src, g0, g1, [&](const InstView& v, long long lo, long long hi) {
      if (v.skip) return true;
      // the column offsets of a step keep 16-byte alignment; Y's base must too
      const bool ybad = (reinterpret_cast<uintptr_t>(v.Y) & 15u) != 0;
      if (ybad && lane == 0) atomicOr(&v.ctl->flags, FLAG_BAD_LAYOUT);
      Walk<C, D> wk;
      wk.start(v, lo);
      for (long long s = lo; s < hi; ++s) {
        if (!mbar_wait_bounded(&cfull[slot], ph, kWaitLimitNs)) {
          atomicOr(&v.ctl->flags, FLAG_TIMEOUT);
          return false;
        }
        if (lane < C::COLVALS / 4) {
          const float* base = ring + slot * C::NW * C::COLVALS + 4 * lane;
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int w = 0; w < C::NW; ++w) {
            if (w < wk.W) {
              const float4 x = *reinterpret_cast<const float4*>(base + w * C::COLVALS);
              sum.x += x.x; sum.y += x.y; sum.z += x.z; sum.w += x.w;
            }
          }
          if (!ybad) red_add_v4_f32(v.Y + (long long)wk.xcol() * D + 4 * lane, sum.x, sum.y, sum.z, sum.w);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&cempty[slot]);
        wk.advance();
        if (++slot == C::RING) {
          slot = 0;
          ph ^= 1u;
        }
      }
      return true;
    });
    return;
  }

  // ---------------------------------------------------------------- consumers
  using Unp = Unpack<ST, C::CPT, C::LOADB>;
  using Vec = typename Unp::V;
  const int rg = lane >> 2;
  const int cg = lane & 3;
  int& st = pp.st;
  int& slot = pp.slot;
  uint32_t& ph = pp.ph;
  uint32_t& cph = pp.cph;
  long long& it = pp.it;  // steps consumed by this CTA so far (all segments and calls)
  uint32_t roff = 0;      // resident modes: dense offset of the current step

  for_segments(src, g0, g1, [&](const InstView& v, long long lo, long long hi) {
    if (v.skip) return true;
    const int n = v.g.n;
    const float* scale =
        (ST == NSRGS_FP8E4M3) ? reinterpret_cast<const float*>(v.packed + v.g.off_scale) : nullptr;
    float xr[C::RT][D];    // X rows of the thread's RT scalar rows (times s_i for FP8)
    float racc[C::RT][D];  // row partials
    const int nrows = n * D;
    auto load_rows = [&](int bb) {
#pragma unroll
      for (int rt = 0; rt < C::RT; ++rt) {
        const int row = bb * C::RS + (warp * 8 + rg) * C::RT + rt;
        float s = 1.f;
        if (ST == NSRGS_FP8E4M3 && row < nrows) s = scale[row / D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          xr[rt][k] = (row < nrows) ? v.X[(long long)row * D + k] * s : 0.f;
          racc[rt][k] = 0.f;
        }
      }
    };
    auto flush_rows = [&](int bb) {
#pragma unroll
      for (int r = 0; r < C::RT; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float x = racc[r][k];
          x += __shfl_xor_sync(0xffffffffu, x, 1);
          x += __shfl_xor_sync(0xffffffffu, x, 2);
          racc[r][k] = x;
        }
      if (cg == 0) {
#pragma unroll
        for (int rt = 0; rt < C::RT; ++rt) {
          const int row = bb * C::RS + (warp * 8 + rg) * C::RT + rt;
          if (row < nrows) {
            const float s = (ST == NSRGS_FP8E4M3) ? scale[row / D] : 1.f;
#pragma unroll
            for (int k = 0; k < D; ++k) red_add_f32(v.Y + (long long)row * D + k, racc[rt][k] * s);
          }
        }
      }
    };

    Walk<C, D> wk;
    wk.start(v, lo);
    load_rows(wk.b);
    for (long long s = lo; s < hi; ++s, ++it) {
      if (!mbar_wait_bounded(&full[st], ph, kWaitLimitNs)) {
        atomicOr(&v.ctl->flags, FLAG_TIMEOUT);
        return false;
      }
      const uint8_t* stage = resident ? smem + roff : smem + st * C::STAGE_BYTES;
      const uint32_t xoff = resident ? (uint32_t)wk.W * C::WB : (uint32_t)C::STAGE_A;
      if (resident) roff += (uint32_t)wk.W * C::WB + C::STAGE_X;
      float cacc[C::NV];
#pragma unroll
      for (int k = 0; k < C::NV; ++k) cacc[k] = 0.f;
      const bool active = warp < wk.W;
      if (active) {
        Vec raw[C::RT];
#pragma unroll
        for (int rt = 0; rt < C::RT; ++rt)
          raw[rt] = *reinterpret_cast<const Vec*>(stage + warp * C::WB + (rt * 32 + lane) * C::LOADB);
        float xc[C::NV];
        if constexpr (C::NV % 4 == 0) {
          const float4* xs = reinterpret_cast<const float4*>(stage + xoff) + cg * (C::NV / 4);
#pragma unroll
          for (int k = 0; k < C::NV / 4; ++k) {
            const float4 t = xs[k];
            xc[4 * k + 0] = t.x; xc[4 * k + 1] = t.y; xc[4 * k + 2] = t.z; xc[4 * k + 3] = t.w;
          }
        } else {
          const float2* xs = reinterpret_cast<const float2*>(stage + xoff) + cg * (C::NV / 2);
#pragma unroll
          for (int k = 0; k < C::NV / 2; ++k) {
            const float2 t = xs[k];
            xc[2 * k + 0] = t.x; xc[2 * k + 1] = t.y;
          }
        }
        // Packed two-wide FMAs (FP32): a row partial's D sums in pairs of k (they
        // share the stored value), the column partials of columns cc, cc + 1 in pairs
        // (they share the X row value).  Every accumulator still sums in the same
        // order (row partials over cc, column partials over rt), so the results are
        // those of scalar fmaf; the FMA instructions drop by about 40% at d = 3.  FP32
        // at n = 10^4, d = 3: 0.2735 -> 0.2656 ms per pass of the fused loop.  BF16
        // measured the same either way and FP8 a little slower (at 168 registers the
        // pairs spill there), so those keep scalar fmaf.
        if constexpr (ST != NSRGS_F32) {
#pragma unroll
          for (int rt = 0; rt < C::RT; ++rt) {
            float av[C::CPT];
            Unp::run(raw[rt], av);
#pragma unroll
            for (int cc = 0; cc < C::CPT; ++cc) {
#pragma unroll
              for (int k = 0; k < D; ++k) {
                racc[rt][k] = fmaf(av[cc], xc[cc * D + k], racc[rt][k]);
                cacc[cc * D + k] = fmaf(av[cc], xr[rt][k], cacc[cc * D + k]);
              }
            }
          }
        } else {
#pragma unroll
        for (int rt = 0; rt < C::RT; ++rt) {
          float av[C::CPT];
          Unp::run(raw[rt], av);
#pragma unroll
          for (int cc = 0; cc < C::CPT; ++cc) {
#pragma unroll
            for (int k = 0; k + 1 < D; k += 2)
              fma2(racc[rt][k], racc[rt][k + 1], av[cc], av[cc], xc[cc * D + k], xc[cc * D + k + 1], racc[rt][k],
                   racc[rt][k + 1]);
            if constexpr (D % 2 == 1) racc[rt][D - 1] = fmaf(av[cc], xc[cc * D + D - 1], racc[rt][D - 1]);
          }
#pragma unroll
          for (int cc = 0; cc + 1 < C::CPT; cc += 2)
#pragma unroll
            for (int k = 0; k < D; ++k)
              fma2(cacc[cc * D + k], cacc[(cc + 1) * D + k], av[cc], av[cc + 1], xr[rt][k], xr[rt][k],
                   cacc[cc * D + k], cacc[(cc + 1) * D + k]);
          if constexpr (C::CPT % 2 == 1) {
#pragma unroll
            for (int k = 0; k < D; ++k)
              cacc[(C::CPT - 1) * D + k] = fmaf(av[C::CPT - 1], xr[rt][k], cacc[(C::CPT - 1) * D + k]);
          }
        }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);  // stage fully read (values consumed above)
      if (++st == C::NSTAGE) {
        st = 0;
        ph ^= 1u;
      }

      // column partials: sum over the 8 rg lanes -> ring slot -> reducer warp
      if constexpr (C::SMEM_RED) {
        // thread (rg, cg) holds ring positions cg*NV .. cg*NV + NV - 1 of row rg
        float* scr = reinterpret_cast<float*>(smem + C::OFF_SCR) + warp * C::SCR_FLOATS;
        float4* dst = reinterpret_cast<float4*>(scr + rg * C::SCR_STRIDE + cg * C::NV);
#pragma unroll
        for (int q = 0; q < C::NV / 4; ++q)
          dst[q] = make_float4(cacc[4 * q], cacc[4 * q + 1], cacc[4 * q + 2], cacc[4 * q + 3]);
        __syncwarp();
        if (it >= C::RING && !mbar_wait_bounded(&cempty[slot], cph ^ 1u, kWaitLimitNs)) {
          atomicOr(&v.ctl->flags, FLAG_TIMEOUT);
          return false;
        }
        if (active && lane < C::COLVALS / 4) {
          float4 sum = reinterpret_cast<const float4*>(scr)[lane];
#pragma unroll
          for (int r = 1; r < 8; ++r) {
            const float4 t = reinterpret_cast<const float4*>(scr + r * C::SCR_STRIDE)[lane];
            sum.x += t.x; sum.y += t.y; sum.z += t.z; sum.w += t.w;
          }
          reinterpret_cast<float4*>(ring + (slot * C::NW + warp) * C::COLVALS)[lane] = sum;
        }
      } else {
        int col0 = 0;
        bool owner = true;
        RedLevel<C::NV, D, 0>::run(cacc, lane, col0, owner);
        constexpr int NF = RedLevel<C::NV, D, 0>::kFinal;
        if (it >= C::RING && !mbar_wait_bounded(&cempty[slot], cph ^ 1u, kWaitLimitNs)) {
          atomicOr(&v.ctl->flags, FLAG_TIMEOUT);
          return false;
        }
        if (owner && active) {
          float* cb = ring + (slot * C::NW + warp) * C::COLVALS + (cg * C::CPT + col0) * D;
#pragma unroll
          for (int k = 0; k < NF; ++k) cb[k] = cacc[k];
        }
      }
      __syncwarp();  // ring written (and the scratch read) before the slot is handed over
      if (lane == 0) mbar_arrive(&cfull[slot]);
      if (++slot == C::RING) {
        slot = 0;
        cph ^= 1u;
      }

      const int bcur = wk.b;
      if (wk.advance()) {
        flush_rows(bcur);
        if (s + 1 < hi) load_rows(wk.b);
      }
    }
    if (wk.q != 0) flush_rows(wk.b);
    return true;
  });
}

// One launch over all steps of `src`, split evenly over the CTAs.
template <int D, int ST, class Src>
__device__ __forceinline__ void panel_stream_body(const Src& src, long long total_steps) {
  const long long g0 = total_steps * blockIdx.x / gridDim.x;
  const long long g1 = total_steps * (blockIdx.x + 1) / gridDim.x;
  if (g0 >= g1) return;
  if (threadIdx.x == 0) panel_init_barriers<D, ST>();
  __syncthreads();
  PanelPipe pp;
  panel_stream_range<D, ST>(src, g0, g1, pp, RES_RING);
}

}  // namespace nsrgs

// Packing of the measurement matrix A into the layouts the iteration streams.
//
// Model (§2.2, eq. (4)): A is symmetric with d x d blocks, A_ji = A_ij^T and
// A_ii = I_d.  The symmetric layouts keep only the strict block-upper triangle
// (each stored block feeds both Y_i += A_ij X_j and Y_j += A_ij^T X_i); the
// dense layout keeps the whole matrix with its diagonal blocks zeroed, so the
// plain product A_off X needs no special case.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "src.cuh"

namespace nsrgs {

static int storage_elem_bytes(int storage) {
  switch (storage) {
    case NSRGS_F32: return 4;
    case NSRGS_BF16: return 2;
    case NSRGS_FP8E4M3: return 1;
    default: return 0;
  }
}

bool make_panel_geom(int n, int d, int storage, PanelGeom* g) {
  if (d < 1 || d > 8 || n < 2) return false;
  int E = storage_elem_bytes(storage);
  if (E == 0) return false;
  if (d > 4 && storage == NSRGS_FP8E4M3) return false;
  PanelGeom G{};
  G.n = n;
  G.D = d;
  G.storage = storage;
  G.E = E;
  G.RT = panel_rt(d, storage);
  G.LOADB = panel_loadb(d, storage);
  G.CPT = G.LOADB / E;
  G.SC = 4 * G.CPT;
  G.NW = panel_nw(d, storage);
  G.RS = G.NW * 8 * G.RT;
  if (G.RS % d != 0) return false;
  G.SB = G.RS / d;
  G.WROWS = 8 * G.RT;
  G.WB = G.WROWS * G.SC * E;
  G.nslabs = (n + G.SB - 1) / G.SB;
  long long steps = 0, bytes = 0;
  for (int b = 0; b < G.nslabs; ++b) {
    long long S = slab_steps(G, b);
    steps += S;
    bytes += panel_step_offset(G, b, S);
  }
  G.total_steps = steps;
  G.panel_bytes = bytes;
  G.off_step_start = 0;
  G.off_byte_off = 8LL * (G.nslabs + 1);
  G.off_scale = G.off_byte_off + 8LL * (G.nslabs + 1);
  long long hdr = G.off_scale + (storage == NSRGS_FP8E4M3 ? 4LL * n : 0);
  G.header_bytes = (hdr + 255) / 256 * 256;
  *g = G;
  return true;
}

static void panel_tables(const PanelGeom& G, std::vector<long long>& tab) {
  tab.assign(2 * (G.nslabs + 1), 0);
  long long s = 0, off = 0;
  for (int b = 0; b <= G.nslabs; ++b) {
    tab[b] = s;
    tab[G.nslabs + 1 + b] = off;
    if (b < G.nslabs) {
      long long S = slab_steps(G, b);
      s += S;
      off += panel_step_offset(G, b, S);
    }
  }
}

// FP8 scales: s_i = max_{j > i} max |A_ij| / 448 (1 when the row is all zero).
template <class Src>
__global__ void fp8_scale_kernel(Src src, int n, int d, float* scale) {
  int i = blockIdx.x;
  long long N = (long long)n * d;
  float m = 0.f;
  for (long long c = (long long)(i + 1) * d + threadIdx.x; c < N; c += blockDim.x)
    for (int a = 0; a < d; ++a) m = fmaxf(m, fabsf(src((long long)i * d + a, c)));
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) scale[i] = (m > 0.f) ? m / 448.f : 1.f;
  }
}

// One CTA per step: writes the step's stored warp slices.
template <class Src>
__global__ void pack_panel_kernel(Src src, PanelGeom g, uint8_t* packed) {
  const long long* step_start = (const long long*)(packed + g.off_step_start);
  const long long* byte_off = (const long long*)(packed + g.off_byte_off);
  const float* scale = (const float*)(packed + g.off_scale);
  long long gs = blockIdx.x + (long long)blockIdx.y * gridDim.x;
  if (gs >= g.total_steps) return;
  int lo = 0, hi = g.nslabs - 1;
  while (lo < hi) {  // last slab whose first step <= gs
    int mid = (lo + hi + 1) >> 1;
    if (step_start[mid] <= gs) lo = mid; else hi = mid - 1;
  }
  int b = lo;
  long long q = gs - step_start[b];
  int W = panel_warps(g, b, q);
  uint8_t* dst = packed + g.header_bytes + byte_off[b] + panel_step_offset(g, b, q);
  long long elems = (long long)W * g.WB / g.E;
  long long row0 = (long long)b * g.SB * g.D;
  long long col0 = (long long)b * g.SB * g.D + q * g.SC;
  int per_load = g.LOADB / g.E;
  for (long long e = threadIdx.x; e < elems; e += blockDim.x) {
    // e -> (w, rt, lane, cc) in the order [w][rt][lane][cc]
    int cc = (int)(e % per_load);
    long long t = e / per_load;
    int lane = (int)(t % 32);
    t /= 32;
    int rt = (int)(t % g.RT);
    int w = (int)(t / g.RT);
    int rg = lane >> 2, cg = lane & 3;
    long long r = (long long)w * g.WROWS + rg * g.RT + rt;
    long long c = (long long)cg * g.CPT + cc;
    float v = src(row0 + r, col0 + c);
    if (g.storage == NSRGS_F32) {
      ((float*)dst)[e] = v;
    } else if (g.storage == NSRGS_BF16) {
      ((__nv_bfloat16*)dst)[e] = __float2bfloat16_rn(v);
    } else {
      long long i = (row0 + r) / g.D;
      float s = (i < g.n) ? scale[i] : 1.f;
      ((__nv_fp8_storage_t*)dst)[e] = __nv_cvt_float_to_fp8(v / s, __NV_SATFINITE, __NV_E4M3);
    }
  }
}

__device__ __forceinline__ void store_as(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_as(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Dense layouts: row pitch = round_up(nd, 4) floats (float32) or round_up(nd, 64)
// bfloat16 values (whole 128-byte rows for the tensor-core stream); diagonal
// blocks zeroed.
template <class Src, class T>
__global__ void pack_dense_kernel(Src src, int n, int d, int pitch, T* out) {
  long long N = (long long)n * d;
  long long total = N * pitch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e / pitch, c = e % pitch;
    float v = 0.f;
    if (c < N) {
      long long i = r / d, j = c / d;
      if (i < j) v = src(r, c);
      else if (i > j) v = src(c, r);  // A_ij = A_ji^T: element (r, c) = (c, r) of the upper part
    }
    store_as(out + e, v);
  }
}

long long dense_pitch(int n, int d) { return ((long long)n * d + 3) / 4 * 4; }
long long dense_bf16_pitch(int n, int d);
bool tc_sym_supported(int d);
template <class Src>
cudaError_t tc_sym_pack(Src src, int n, int d, bool f8, void* packed, cudaStream_t st);
long long tc_sym8_scale_offset(int n, int d);
bool fs_sym_supported(int d);
template <class Src>
cudaError_t fs_sym_pack(Src src, int n, int d, void* packed, cudaStream_t st);

template <class Src>
static nsrgs_status pack_any(Src src, int n, int d, int storage, void* packed, cudaStream_t st) {
  if (storage == NSRGS_DENSE_F32) {
    long long pitch = dense_pitch(n, d);
    pack_dense_kernel<<<4 * num_sms(), 256, 0, st>>>(src, n, d, (int)pitch, (float*)packed);
    NSRGS_CUDA_TRY(cudaGetLastError());
    return NSRGS_OK;
  }
  if (storage == NSRGS_DENSE_BF16) {
    long long pitch = dense_bf16_pitch(n, d);
    pack_dense_kernel<<<4 * num_sms(), 256, 0, st>>>(src, n, d, (int)pitch, (__nv_bfloat16*)packed);
    NSRGS_CUDA_TRY(cudaGetLastError());
    return NSRGS_OK;
  }
  {  // tile layouts (also the SE(d) form's augmented blocks above D = 8)
    if (tile_storage(storage, d) && !tile_fp8(storage)) {
      NSRGS_CUDA_TRY(tc_sym_pack(src, n, d, false, packed, st));
      return NSRGS_OK;
    }
    if (tile_storage(storage, d)) {  // FP8: block-row scales first, behind the tiles
      fp8_scale_kernel<<<n, 256, 0, st>>>(src, n, d, (float*)((uint8_t*)packed + tc_sym8_scale_offset(n, d)));
      NSRGS_CUDA_TRY(cudaGetLastError());
      NSRGS_CUDA_TRY(tc_sym_pack(src, n, d, true, packed, st));
      return NSRGS_OK;
    }
    if (storage == NSRGS_F32 && fs_sym_supported(d)) {
      NSRGS_CUDA_TRY(fs_sym_pack(src, n, d, packed, st));
      return NSRGS_OK;
    }
  }
  PanelGeom g;
  if (!make_panel_geom(n, d, storage, &g)) {
    set_error("symmetric storage needs F32 (any d <= 64), BF16 with any d <= 64, FP8 with d <= 4 or 8 < d <= 64; use NSRGS_DENSE_F32");
    return NSRGS_ERR_UNSUPPORTED;
  }
  std::vector<long long> tab;
  panel_tables(g, tab);
  NSRGS_CUDA_TRY(cudaMemcpyAsync(packed, tab.data(), tab.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
  if (storage == NSRGS_FP8E4M3) {
    fp8_scale_kernel<<<n, 256, 0, st>>>(src, n, d, (float*)((uint8_t*)packed + g.off_scale));
    NSRGS_CUDA_TRY(cudaGetLastError());
  }
  long long S = g.total_steps;
  dim3 grid((unsigned)std::min<long long>(S, 65535), (unsigned)((S + 65534) / 65535));
  pack_panel_kernel<<<grid, 256, 0, st>>>(src, g, (uint8_t*)packed);
  NSRGS_CUDA_TRY(cudaGetLastError());
  // cudaMemcpyAsync from pageable memory has staged `tab` before returning.
  return NSRGS_OK;
}

bool bcsr_storage(int storage);
cudaError_t bcsr_pack_upper(const float* upper, int n, int d, int storage, void* packed, cudaStream_t st);
cudaError_t bcsr_pack_dense(const float* A, int n, int d, int storage, void* packed, cudaStream_t st);

static nsrgs_status check_bcsr_d(int d) {
  if (d > 8) {
    set_error("block-sparse storage covers d <= 8");
    return NSRGS_ERR_UNSUPPORTED;
  }
  return NSRGS_OK;
}

nsrgs_status pack_upper_impl(const float* upper, int n, int d, int storage, void* packed, cudaStream_t st) {
  if (bcsr_storage(storage)) {
    nsrgs_status s = check_bcsr_d(d);
    if (s != NSRGS_OK) return s;
    NSRGS_CUDA_TRY(bcsr_pack_upper(upper, n, d, storage, packed, st));
    return NSRGS_OK;
  }
  return pack_any(UpperSrc{upper, n, d}, n, d, storage, packed, st);
}

// SE(d) form: the augmented (d+1)-block matrix in the symmetric panel layout.
nsrgs_status pack_se_impl(const float* upper_a, const float* upper_c, int n, int d, float kappa, int storage,
                          void* packed, cudaStream_t st) {
  return pack_any(SeAugSrc{upper_a, upper_c, n, d, sqrtf(kappa)}, n, d + 1, storage, packed, st);
}

nsrgs_status pack_dense_impl(const float* A, int n, int d, int storage, void* packed, cudaStream_t st) {
  if (bcsr_storage(storage)) {
    nsrgs_status s = check_bcsr_d(d);
    if (s != NSRGS_OK) return s;
    NSRGS_CUDA_TRY(bcsr_pack_dense(A, n, d, storage, packed, st));
    return NSRGS_OK;
  }
  return pack_any(DenseSrc{A, n, d}, n, d, storage, packed, st);
}

}  // namespace nsrgs

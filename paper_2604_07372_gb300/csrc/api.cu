// C ABI of libnsrgs: argument checks, workspace layout, the spectral
// initialisation sequence, one iteration, and the graph-replayed solve.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace nsrgs {

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

int num_sms() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

// ------------------------------------------------- kernels in other units
nsrgs_status pack_upper_impl(const float*, int, int, int, void*, cudaStream_t);
nsrgs_status pack_dense_impl(const float*, int, int, int, void*, cudaStream_t);
nsrgs_status pack_se_impl(const float*, const float*, int, int, float, int, void*, cudaStream_t);
cudaError_t se_launch(int what, int d, const float* X, float* t, const float* Xa0, float* Ya, float* Xa1, int n,
                      float eta, float eta_t, float kappa, int K, double tol, Ctl* ctl, float* Xout,
                      cudaStream_t st);
cudaError_t se_prepare(int d);
long long dense_pitch(int n, int d);
cudaError_t stream_panel(const void* packed, const PanelGeom& g, const float* X, float* Y, Ctl* ctl,
                         const int* skip, cudaStream_t st);
cudaError_t stream_dense(const void* packed, int n, int d, const float* X, float* Y, const int* skip,
                         cudaStream_t st);
cudaError_t stream_panel_prepare(const PanelGeom& g);
cudaError_t iterate_panel_loop(const void* packed, const PanelGeom& g, float* X0, float* X1, float* Y, float eta, int K,
                               int safeguard, int T, double tol, Ctl* ctl, const int* skip, cudaStream_t st);

int reduce_grid(long long rows);
cudaError_t launch_epilogue(const float*, float*, float*, int, int, float, int, int, double, Ctl*, double*,
                            cudaStream_t);
cudaError_t launch_gpm_epilogue(const float*, float*, float*, int, int, double, Ctl*, cudaStream_t);
cudaError_t launch_spec_v0(float*, long long, int, double*, cudaStream_t);
cudaError_t launch_spec_gram(const float*, float*, float*, long long, int, float, int, int, const SpecScratch&,
                             Ctl*, cudaStream_t);
cudaError_t launch_spec_update(const float*, const float*, float*, long long, int, const SpecScratch&, double, int,
                               Ctl*, cudaStream_t);
cudaError_t launch_polar_blocks(const float*, float*, int, int, cudaStream_t);
cudaError_t launch_dF(const float*, const float*, long long, int, const SpecScratch&, Ctl*, cudaStream_t);
cudaError_t launch_copy_out(const float*, const float*, float*, long long, const Ctl*, cudaStream_t);
cudaError_t launch_select_copy(const float*, const float*, float*, long long, const Ctl*, cudaStream_t);
cudaError_t generic_prepare(int d);
long long dense_bf16_pitch(int n, int d);
bool tc_dense_supported(int d);
cudaError_t tc_dense_prepare(int d);
cudaError_t tc_dense_product(const void* packed, int n, int d, const float* X, __nv_bfloat16* XT, float* Y, Ctl* ctl,
                             const int* skip, cudaStream_t st);
cudaError_t tc_dense_tune(const void* packed, int n, int d, __nv_bfloat16* XT, float* Y, Ctl* ctl, const int* skip,
                          cudaStream_t st);
int tc_dense_splits(int n, int d);
bool bcsr_storage(int storage);
long long bcsr_bytes(int n, int d, int storage, long long nnzb);
cudaError_t bcsr_stream(const void* packed, int n, int d, int storage, const float* X, float* Y, const int* skip,
                        Ctl* ctl, cudaStream_t st);
cudaError_t bcsr_count_upper(const float* upper, int n, int d, unsigned long long* d_total, cudaStream_t st);
cudaError_t bcsr_count_dense(const float* A, int n, int d, unsigned long long* d_total, cudaStream_t st);
bool tc_sym_supported(int d);
long long tc_sym_bytes(int n, int d);
long long tc_sym8_bytes(int n, int d);
long long tc_sym8_xt_bytes(int n, int d);
cudaError_t tc_sym_prepare(int d, bool f8);
cudaError_t tc_sym_product(const void* packed, int n, int d, bool f8, const float* X, uint8_t* xt, float* Y,
                           Ctl* ctl, const int* skip, cudaStream_t st);

// Tile-upper tensor-core storage (tile_storage in common.cuh).
static bool tile_upper(int storage, int d) { return tile_storage(storage, d); }
bool fs_sym_supported(int d);
long long fs_sym_bytes(int n, int d);
long long fs_sym_xt_bytes(int n, int d);
cudaError_t fs_sym_prepare(int d);
cudaError_t fs_sym_product(const void* packed, int n, int d, const float* X, float* xt, float* Y, Ctl* ctl,
                           const int* skip, cudaStream_t st);
size_t obj_partials_doubles(int n, int D);
cudaError_t launch_objective(const float* Xc, const float* Yc, const float* Xp, float* Yp, int n, int D,
                             double rel_tol, const ObjScratch& o, Ctl* ctl, cudaStream_t st);
cudaError_t launch_norm2(const void* packed, int n, int d, int storage, const PanelGeom& g, const ObjScratch& o,
                         Ctl* ctl, cudaStream_t st);

constexpr int kMaxReduceGrid = 512;
constexpr int kMaxSmallD = 8;

// ---------------------------------------------------------- workspace map
struct Workspace {
  Ctl* ctl;
  float* X[2];
  float* Y;
  float* W;
  SpecScratch s;
  ObjScratch obj;
  __nv_bfloat16* XT;  // X^T in bfloat16 for the tensor-core stream (d >= 16 only)
  size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static Workspace map_workspace(void* base, int n, int d) {
  Workspace w{};
  size_t off = 0;
  uint8_t* p = reinterpret_cast<uint8_t*>(base);
  auto take = [&](size_t bytes) {
    uint8_t* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  const size_t vec = (size_t)xpad_rows(n, d) * d * sizeof(float);
  w.ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  w.X[0] = reinterpret_cast<float*>(take(vec));
  w.X[1] = reinterpret_cast<float*>(take(vec));
  w.Y = reinterpret_cast<float*>(take(vec));
  w.W = reinterpret_cast<float*>(take(vec));
  const size_t dd = (size_t)d * d * sizeof(double);
  w.s.WW = reinterpret_cast<double*>(take(dd));
  w.s.H = reinterpret_cast<double*>(take(dd));
  w.s.Rinv = reinterpret_cast<double*>(take(dd));
  w.s.M = reinterpret_cast<double*>(take(dd));
  w.s.Q = reinterpret_cast<double*>(take(dd));
  w.s.scal = reinterpret_cast<double*>(take(8 * sizeof(double)));
  w.s.partials = reinterpret_cast<double*>(take((size_t)kMaxReduceGrid * 2 * dd));
  w.obj.scal = reinterpret_cast<double*>(take(OBJ_NSCAL * sizeof(double)));
  w.obj.Gprev = reinterpret_cast<double*>(take(dd));
  w.obj.total = reinterpret_cast<double*>(take(dd + 3 * sizeof(double)));
  w.obj.partials = reinterpret_cast<double*>(take(obj_partials_doubles(n, d) * sizeof(double)));
  w.obj.Yprev = reinterpret_cast<float*>(take(vec));
  if (d > 8) {
    // X^T: bfloat16 row-major for the dense tensor-core stream, swizzled bfloat16 tiles
    // (or two sets of E4M3 hi / lo planes) for the tile-upper tensor-core stream,
    // float32 64-row tiles for the float32 tile stream
    long long a = fs_sym_xt_bytes(n, d);
    const long long c = tc_sym8_xt_bytes(n, d);
    a = a > c ? a : c;
    if (d >= 16) {
      const long long b = (long long)d * dense_bf16_pitch(n, d) * 2;
      a = a > b ? a : b;
    }
    w.XT = reinterpret_cast<__nv_bfloat16*>(take((size_t)a));
  }
  w.bytes = off;
  return w;
}

// ------------------------------------------------------------- checks
static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static nsrgs_status check_nd(int n, int d) {
  NSRGS_CHECK_ARG(n >= 2, "n must be >= 2");
  NSRGS_CHECK_ARG(d >= 1 && d <= 64, "d must be in [1, 64]");
  NSRGS_CHECK_ARG((long long)n * d <= (1LL << 30) / 64, "n*d too large");
  return NSRGS_OK;
}

// Every d in [1, 64] has per-block kernels: registers for d <= 8, shared memory
// (generic.cu) above; their launch attributes are set here, outside any capture.
static nsrgs_status check_small_d(int d) {
  if (d > kMaxSmallD) NSRGS_CUDA_TRY(generic_prepare(d));
  return NSRGS_OK;
}

static nsrgs_status check_A(const nsrgs_A* A, PanelGeom* g) {
  NSRGS_CHECK_ARG(A != nullptr, "A is null");
  nsrgs_status s = check_nd(A->n, A->d);
  if (s != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(A->packed != nullptr && aligned16(A->packed), "A->packed must be a 16-byte aligned device pointer");
  if (A->storage == NSRGS_DENSE_F32) return NSRGS_OK;
  if (A->storage == NSRGS_DENSE_BF16) {
    if (!tc_dense_supported(A->d)) {
      set_error("NSRGS_DENSE_BF16 (tensor-core stream) covers d in {16, 32, 64}");
      return NSRGS_ERR_UNSUPPORTED;
    }
    NSRGS_CUDA_TRY(tc_dense_prepare(A->d));
    return NSRGS_OK;
  }
  if (bcsr_storage(A->storage)) {
    if (A->d > 8) {
      set_error("block-sparse storage covers d <= 8");
      return NSRGS_ERR_UNSUPPORTED;
    }
    return NSRGS_OK;
  }
  if (tile_upper(A->storage, A->d)) {
    NSRGS_CUDA_TRY(tc_sym_prepare(A->d, tile_fp8(A->storage)));
    return NSRGS_OK;
  }
  NSRGS_CHECK_ARG(A->storage >= NSRGS_F32 && A->storage <= NSRGS_FP8E4M3, "unknown storage");
  if (A->storage == NSRGS_F32 && fs_sym_supported(A->d)) {
    NSRGS_CUDA_TRY(fs_sym_prepare(A->d));
    return NSRGS_OK;
  }
  if (!make_panel_geom(A->n, A->d, A->storage, g)) {
    set_error("symmetric storage needs F32 (any d <= 64), BF16 with any d <= 64, FP8 with d <= 4 or 8 < d <= 64; use NSRGS_DENSE_F32");
    return NSRGS_ERR_UNSUPPORTED;
  }
  NSRGS_CUDA_TRY(stream_panel_prepare(*g));
  return NSRGS_OK;
}

static nsrgs_status check_ws(void* ws, size_t ws_bytes, int n, int d) {
  NSRGS_CHECK_ARG(ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0,
                  "workspace must be a 256-byte aligned device pointer");
  const size_t need = map_workspace(nullptr, n, d).bytes;
  if (ws_bytes < need) {
    set_error("workspace smaller than nsrgs_workspace_bytes(n, d)");
    return NSRGS_ERR_NOMEM;
  }
  return NSRGS_OK;
}

// ---------------------------------------------------------------- pieces
static cudaError_t stream_AX(const nsrgs_A* A, const PanelGeom& g, const float* X, const Workspace& w,
                             const int* skip, cudaStream_t st) {
  if (A->storage == NSRGS_DENSE_F32) return stream_dense(A->packed, A->n, A->d, X, w.Y, skip, st);
  if (A->storage == NSRGS_DENSE_BF16) return tc_dense_product(A->packed, A->n, A->d, X, w.XT, w.Y, w.ctl, skip, st);
  if (tile_upper(A->storage, A->d))
    return tc_sym_product(A->packed, A->n, A->d, tile_fp8(A->storage), X, reinterpret_cast<uint8_t*>(w.XT),
                          w.Y, w.ctl, skip, st);
  if (A->storage == NSRGS_F32 && fs_sym_supported(A->d))
    return fs_sym_product(A->packed, A->n, A->d, X, reinterpret_cast<float*>(w.XT), w.Y, w.ctl, skip, st);
  if (bcsr_storage(A->storage)) return bcsr_stream(A->packed, A->n, A->d, A->storage, X, w.Y, skip, w.ctl, st);
  return stream_panel(A->packed, g, X, w.Y, w.ctl, skip, st);
}

// Tensor-core storage: pick the split-K for this shape once (timed, outside any
// capture).  Clobbers Y and the control block; callers reset both afterwards.
static cudaError_t maybe_tune(const nsrgs_A* A, const Workspace& w, cudaStream_t st) {
  if (A->storage != NSRGS_DENSE_BF16) return cudaSuccess;
  if (tc_dense_splits(A->n, A->d) > 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st);
  if (e != cudaSuccess) return e;
  return tc_dense_tune(A->packed, A->n, A->d, w.XT, w.Y, w.ctl, &w.ctl->stop, st);
}

// Resets the control block and zeroes Y and the padding of the X buffers.
static cudaError_t reset_ws(const Workspace& w, int n, int d, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.obj.scal, 0, OBJ_NSCAL * sizeof(double), st)) != cudaSuccess) return e;
  const size_t vec = (size_t)xpad_rows(n, d) * d * sizeof(float);
  const size_t body = (size_t)n * d * d * sizeof(float);
  if ((e = cudaMemsetAsync(w.Y, 0, vec, st)) != cudaSuccess) return e;
  for (int k = 0; k < 2; ++k)
    if ((e = cudaMemsetAsync(reinterpret_cast<uint8_t*>(w.X[k]) + body, 0, vec - body, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Subspace iteration for the top-d eigenvectors of A, then the exact blockwise
// sign: X0 = sgn_n(V) (Algorithm 2's spectral initialisation).  The passes
// iterate on A_off + cI, starting with c = 1 (A itself); at convergence the
// algebraic top-d test (spec_shift_after) either accepts the subspace or
// restarts from V^0 with a larger c inside the same pass budget.
// Leaves X0 in `out` (which may be w.X[0]); uses X[0], X[1], Y, W.
static cudaError_t enqueue_spectral(const nsrgs_A* A, const PanelGeom& g, const Workspace& w, int max_iters,
                                    double tol, float* out, cudaStream_t st) {
  const int n = A->n, d = A->d;
  const long long rows = (long long)n * d;
  // the tensor-core streams round V (bfloat16, or E4M3 hi / lo planes): their passes
  // may also stop at the residual floor that rounding sets, and their float64-free
  // Gram and update (float32 inner products over 64-row chunks, about 1e-7 of the
  // terms) stay far below that floor
  // (mode 3: the float32 tile stream, whose long float32 sums floor near 1e-6)
  const int counted = (A->storage == NSRGS_DENSE_BF16 || tile_upper(A->storage, d))
                          ? 2
                          : ((A->storage == NSRGS_F32 && fs_sym_supported(d)) ? 3 : 1);
  cudaError_t e;
  if ((e = launch_spec_v0(w.X[0], rows, d, w.s.scal + 3, st)) != cudaSuccess) return e;
  // orthonormalise the start: W = V0 (Y is zero), V1 = W chol(W^T W)^{-1}
  if ((e = launch_spec_gram(w.X[0], w.Y, w.W, rows, d, 1.0f, 0, 0, w.s, w.ctl, st)) != cudaSuccess) return e;
  if ((e = launch_spec_update(w.X[0], w.W, w.X[1], rows, d, w.s, tol, 0, w.ctl, st)) != cudaSuccess) return e;
  for (int k = 0; k < max_iters; ++k) {
    const float* V = w.X[(k + 1) & 1];
    float* Vn = w.X[k & 1];
    if ((e = stream_AX(A, g, V, w, &w.ctl->spec_skip, st)) != cudaSuccess) return e;
    if ((e = launch_spec_gram(V, w.Y, w.W, rows, d, 1.0f, 1, counted == 2, w.s, w.ctl, st)) != cudaSuccess) return e;
    if ((e = launch_spec_update(V, w.W, Vn, rows, d, w.s, tol, counted, w.ctl, st)) != cudaSuccess) return e;
  }
  // final basis -> W, then X0 = sgn_n(W)
  if ((e = launch_select_copy(w.X[0], w.X[1], w.W, rows * d, w.ctl, st)) != cudaSuccess) return e;
  return launch_polar_blocks(w.W, out, n, d, st);
}

enum { METHOD_NSRGS = 0, METHOD_GPM = 1, METHOD_NSRGS_OBJECTIVE = 2 };

// On the panel layouts (symmetric storage at d <= 7) the T iterations of
// Algorithm 2 run as ONE persistent launch (A stream, grid barrier, block
// updates, grid barrier, per iteration); at d = 8 the fused kernel would spill the
// block update's 8 x 8 registers, so there each iteration stays a stream launch
// plus an epilogue launch.
static bool fused_loop(const nsrgs_A* A, int method) {
  return method == METHOD_NSRGS && A->d <= 7 &&
         (A->storage == NSRGS_F32 || A->storage == NSRGS_BF16 || A->storage == NSRGS_FP8E4M3);
}

static cudaError_t enqueue_iterations(const nsrgs_A* A, const PanelGeom& g, const Workspace& w, float eta, int T,
                                      int K, double tol, int method, int safeguard, cudaStream_t st,
                                      const cudaEvent_t* ev = nullptr) {
  cudaError_t e;
  if (fused_loop(A, method)) {
    if (T == 0) return cudaSuccess;
    if (ev && (e = cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    e = iterate_panel_loop(A->packed, g, w.X[0], w.X[1], w.Y, eta, K, safeguard, T, tol, w.ctl, &w.ctl->stop, st);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  for (int t = 0; t < T; ++t) {
    const float* Xt = w.X[t & 1];
    float* Xn = w.X[(t + 1) & 1];
    if (ev && (e = cudaEventRecordWithFlags(ev[2 * t], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = stream_AX(A, g, Xt, w, &w.ctl->stop, st)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecordWithFlags(ev[2 * t + 1], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (method == METHOD_GPM) {
      e = launch_gpm_epilogue(Xt, w.Y, Xn, A->n, A->d, tol, w.ctl, st);
    } else if (method == METHOD_NSRGS_OBJECTIVE) {
      // F(X^t) and R^{t-1} from Y = A_off X^t (Xn still holds X^{t-1}); a stop
      // leaves X^t as the result and skips this iteration's update
      e = launch_objective(Xt, w.Y, Xn, w.obj.Yprev, A->n, A->d, tol, w.obj, w.ctl, st);
      if (e == cudaSuccess) e = launch_epilogue(Xt, w.Y, Xn, A->n, A->d, eta, K, safeguard, 0.0, w.ctl, nullptr, st);
    } else {
      e = launch_epilogue(Xt, w.Y, Xn, A->n, A->d, eta, K, safeguard, tol, w.ctl, nullptr, st);
    }
    if (e != cudaSuccess) return e;
  }
  if (method == METHOD_NSRGS_OBJECTIVE) {
    // one more product for F(X^T) and R^{T-1} (skipped after a stop)
    if ((e = stream_AX(A, g, w.X[T & 1], w, &w.ctl->stop, st)) != cudaSuccess) return e;
    if ((e = launch_objective(w.X[T & 1], w.Y, w.X[(T + 1) & 1], w.obj.Yprev, A->n, A->d, tol, w.obj, w.ctl, st)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------ graph cache
struct GraphKey {
  int dev;
  const void* packed;
  int n, d, storage;
  float eta;
  int T, K;
  double tol;
  int init, smax;
  float* X;
  void* ws;
  int timing;
  int method;
  int safeguard;
  bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  int kernel_nodes;
};

static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;  // most recent last
static cudaStream_t g_capture_stream[64] = {};

static cudaError_t capture_stream(int dev, cudaStream_t* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_capture_stream[dev]) {
    cudaError_t e = cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = g_capture_stream[dev];
  return cudaSuccess;
}

// ----------------------------------------------------- kernel timing aid
static int g_timing = 0;
struct TimingState {
  std::vector<cudaEvent_t> ev;  // 2 per iteration (before / after the A stream)
  int last_T = 0;               // pairs recorded by the most recently launched timed graph
  int per_pair = 1;             // iterations inside one timed pair (T for the fused loop)
  int last_nodes = 0;           // kernel nodes of the most recently launched graph
};
static TimingState g_timing_state[64];

static cudaError_t ensure_events(int dev, int T) {
  std::vector<cudaEvent_t>& ev = g_timing_state[dev].ev;
  while ((int)ev.size() < 2 * T) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
  }
  return cudaSuccess;
}

static int count_kernel_nodes(cudaGraph_t graph) {
  size_t num = 0;
  if (cudaGraphGetNodes(graph, nullptr, &num) != cudaSuccess || num == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(num);
  if (cudaGraphGetNodes(graph, nodes.data(), &num) != cudaSuccess) return 0;
  int k = 0;
  for (size_t i = 0; i < num; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

}  // namespace nsrgs

using namespace nsrgs;

extern "C" {

const char* nsrgs_last_error(void) { return get_error(); }

const char* nsrgs_version(void) { return "nsrgs-gb300 0.1 (sm_103a)"; }

size_t nsrgs_packed_bytes(int n, int d, int storage) {
  if (n < 2 || d < 1 || d > 64) return 0;
  if (storage == NSRGS_DENSE_F32) return (size_t)n * d * (size_t)dense_pitch(n, d) * sizeof(float);
  if (storage == NSRGS_DENSE_BF16)
    return tc_dense_supported(d) ? (size_t)n * d * (size_t)dense_bf16_pitch(n, d) * 2 : 0;
  if (tile_upper(storage, d)) return (size_t)(tile_fp8(storage) ? tc_sym8_bytes(n, d) : tc_sym_bytes(n, d));
  if (storage == NSRGS_F32 && fs_sym_supported(d)) return (size_t)fs_sym_bytes(n, d);
  if (bcsr_storage(storage)) return d <= 8 ? (size_t)bcsr_bytes(n, d, storage, (long long)n * (n - 1)) : 0;
  PanelGeom g;
  if (!make_panel_geom(n, d, storage, &g)) return 0;
  return (size_t)(g.header_bytes + g.panel_bytes);
}

size_t nsrgs_workspace_bytes(int n, int d) {
  if (n < 2 || d < 1 || d > 64) return 0;
  return map_workspace(nullptr, n, d).bytes;
}

nsrgs_status nsrgs_bcsr_packed_bytes(const float* src, int src_is_dense, int n, int d, int storage, size_t* bytes,
                                     void* ws, size_t ws_bytes, void* stv) {
  nsrgs_status s = check_nd(n, d);
  if (s != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(bcsr_storage(storage), "storage must be NSRGS_BCSR_F32 or NSRGS_BCSR_BF16");
  NSRGS_CHECK_ARG(d <= 8, "block-sparse storage covers d <= 8");
  NSRGS_CHECK_ARG(src && bytes, "src and bytes must be non-null");
  if ((s = check_ws(ws, ws_bytes, n, d)) != NSRGS_OK) return s;
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, n, d);
  // the count lands in the first 8 bytes of the spectral scalars (8 doubles)
  unsigned long long* total = reinterpret_cast<unsigned long long*>(w.s.scal);
  NSRGS_CUDA_TRY(src_is_dense ? bcsr_count_dense(src, n, d, total, st) : bcsr_count_upper(src, n, d, total, st));
  unsigned long long nnzb = 0;
  NSRGS_CUDA_TRY(cudaMemcpyAsync(&nnzb, total, sizeof(nnzb), cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
  *bytes = (size_t)bcsr_bytes(n, d, storage, (long long)nnzb);
  return NSRGS_OK;
}

nsrgs_status nsrgs_pack_upper(const float* upper, int n, int d, int storage, void* packed, void* st) {
  nsrgs_status s = check_nd(n, d);
  if (s != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(upper && packed && aligned16(packed), "null or misaligned pointer");
  return pack_upper_impl(upper, n, d, storage, packed, (cudaStream_t)st);
}

nsrgs_status nsrgs_pack_dense(const float* A, int n, int d, int storage, void* packed, void* st) {
  nsrgs_status s = check_nd(n, d);
  if (s != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(A && packed && aligned16(packed), "null or misaligned pointer");
  return pack_dense_impl(A, n, d, storage, packed, (cudaStream_t)st);
}

nsrgs_status nsrgs_spectral_init(const nsrgs_A* A, float* X0, int max_iters, double tol, double* residual, void* ws,
                                 size_t ws_bytes, void* stv) {
  PanelGeom g{};
  nsrgs_status s = check_A(A, &g);
  if (s != NSRGS_OK) return s;
  if ((s = check_small_d(A->d)) != NSRGS_OK) return s;
  if ((s = check_ws(ws, ws_bytes, A->n, A->d)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(X0 && aligned16(X0), "X0 must be a 16-byte aligned device pointer");
  NSRGS_CHECK_ARG(max_iters >= 1 && max_iters <= 10000, "max_iters must be in [1, 10000]");
  NSRGS_CHECK_ARG(tol >= 0.0 && isfinite(tol), "tol must be finite and >= 0");
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, A->n, A->d);
  NSRGS_CUDA_TRY(maybe_tune(A, w, st));
  NSRGS_CUDA_TRY(reset_ws(w, A->n, A->d, st));
  NSRGS_CUDA_TRY(enqueue_spectral(A, g, w, max_iters, tol, X0, st));
  Ctl c{};
  NSRGS_CUDA_TRY(cudaMemcpyAsync(&c, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
  if (residual) *residual = c.spec_res;
  if (c.flags & FLAG_BAD_LAYOUT) {
    set_error("the packed A is inconsistent: an index or address left its buffer (access skipped)");
    return NSRGS_ERR_INVALID_ARG;
  }
  if (c.flags & FLAG_TIMEOUT) {
    set_error("a device-side wait timed out");
    return NSRGS_ERR_TIMEOUT;
  }
  if (!c.spec_stop) {
    set_error("spectral initialisation did not reach tol within max_iters");
    return NSRGS_ERR_NOT_CONVERGED;
  }
  return NSRGS_OK;
}

nsrgs_status nsrgs_product(const nsrgs_A* A, const float* X, float* Y, void* ws, size_t ws_bytes, void* stv) {
  PanelGeom g{};
  nsrgs_status s = check_A(A, &g);
  if (s != NSRGS_OK) return s;
  if ((s = check_ws(ws, ws_bytes, A->n, A->d)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(X && Y && aligned16(X) && aligned16(Y), "X/Y must be 16-byte aligned device pointers");
  const size_t bytes = (size_t)A->n * A->d * A->d * sizeof(float);
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, A->n, A->d);
  NSRGS_CUDA_TRY(maybe_tune(A, w, st));
  NSRGS_CUDA_TRY(reset_ws(w, A->n, A->d, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(w.X[0], X, bytes, cudaMemcpyDeviceToDevice, st));
  NSRGS_CUDA_TRY(stream_AX(A, g, w.X[0], w, &w.ctl->stop, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(Y, w.Y, bytes, cudaMemcpyDeviceToDevice, st));
  return NSRGS_OK;
}

nsrgs_status nsrgs_step(const nsrgs_A* A, float eta, int K, const float* X_in, float* X_out, double* upd_norm,
                        void* ws, size_t ws_bytes, void* stv) {
  PanelGeom g{};
  nsrgs_status s = check_A(A, &g);
  if (s != NSRGS_OK) return s;
  if ((s = check_small_d(A->d)) != NSRGS_OK) return s;
  if ((s = check_ws(ws, ws_bytes, A->n, A->d)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(eta > 0.f && isfinite(eta), "eta must be finite and > 0");
  NSRGS_CHECK_ARG(K >= 0 && K <= 64, "K must be in [0, 64]");
  NSRGS_CHECK_ARG(X_in && X_out && aligned16(X_in) && aligned16(X_out), "X_in/X_out must be 16-byte aligned");
  const size_t bytes = (size_t)A->n * A->d * A->d * sizeof(float);
  const uint8_t* a0 = reinterpret_cast<const uint8_t*>(X_in);
  const uint8_t* b0 = reinterpret_cast<const uint8_t*>(X_out);
  NSRGS_CHECK_ARG(a0 + bytes <= b0 || b0 + bytes <= a0, "X_in and X_out overlap");
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, A->n, A->d);
  NSRGS_CUDA_TRY(maybe_tune(A, w, st));
  NSRGS_CUDA_TRY(reset_ws(w, A->n, A->d, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(w.X[0], X_in, bytes, cudaMemcpyDeviceToDevice, st));
  NSRGS_CUDA_TRY(stream_AX(A, g, w.X[0], w, &w.ctl->stop, st));
  NSRGS_CUDA_TRY(launch_epilogue(w.X[0], w.Y, X_out, A->n, A->d, eta, K, 0, 0.0, w.ctl, upd_norm, st));
  return NSRGS_OK;
}

static nsrgs_status solve_impl(const nsrgs_A* A, float eta, int T, int K, double tol, int init,
                               int spectral_max_iters, float* X, nsrgs_info* info, void* ws, size_t ws_bytes,
                               void* stv, int method, int safeguard = 0);

nsrgs_status nsrgs_solve(const nsrgs_A* A, float eta, int T, int K, double tol, int init, int spectral_max_iters,
                         float* X, nsrgs_info* info, void* ws, size_t ws_bytes, void* stv) {
  return solve_impl(A, eta, T, K, tol, init, spectral_max_iters, X, info, ws, ws_bytes, stv, METHOD_NSRGS);
}

nsrgs_status nsrgs_gpm_solve(const nsrgs_A* A, int T, double tol, int init, int spectral_max_iters, float* X,
                             nsrgs_info* info, void* ws, size_t ws_bytes, void* stv) {
  return solve_impl(A, 1.0f, T, 0, tol, init, spectral_max_iters, X, info, ws, ws_bytes, stv, METHOD_GPM);
}

nsrgs_status nsrgs_solve_objective(const nsrgs_A* A, float eta, int T, int K, double rel_tol, int init,
                                   int spectral_max_iters, float* X, nsrgs_info* info, void* ws, size_t ws_bytes,
                                   void* stv) {
  NSRGS_CHECK_ARG(isfinite(rel_tol), "rel_tol must be finite");
  return solve_impl(A, eta, T, K, rel_tol, init, spectral_max_iters, X, info, ws, ws_bytes, stv,
                    METHOD_NSRGS_OBJECTIVE);
}

nsrgs_status nsrgs_solve_ex(const nsrgs_A* A, float eta, int T, int K, const nsrgs_solve_opts* opts, int init,
                            int spectral_max_iters, float* X, nsrgs_info* info, void* ws, size_t ws_bytes, void* stv) {
  NSRGS_CHECK_ARG(opts != nullptr, "opts is null");
  NSRGS_CHECK_ARG(opts->stop_rule == NSRGS_STOP_UPDATE_NORM || opts->stop_rule == NSRGS_STOP_REL_DECREASE,
                  "unknown stop_rule");
  NSRGS_CHECK_ARG(isfinite(opts->tol), "tol must be finite");
  const int method = opts->stop_rule == NSRGS_STOP_REL_DECREASE ? METHOD_NSRGS_OBJECTIVE : METHOD_NSRGS;
  return solve_impl(A, eta, T, K, opts->tol, init, spectral_max_iters, X, info, ws, ws_bytes, stv, method,
                    opts->ns_safeguard ? 1 : 0);
}

nsrgs_status nsrgs_solve_host(const nsrgs_A* A, const void* packed_host, size_t packed_bytes, float eta, int T,
                              int K, double tol, int init, int spectral_max_iters, float* X, float* X_host,
                              nsrgs_info* info, void* ws, size_t ws_bytes, void* stv) {
  NSRGS_CHECK_ARG(A != nullptr && A->packed != nullptr, "A and A->packed must be non-null");
  NSRGS_CHECK_ARG(packed_host && X_host, "packed_host and X_host must be non-null host pointers");
  nsrgs_status s = check_nd(A->n, A->d);
  if (s != NSRGS_OK) return s;
  const int n = A->n, d = A->d;
  // The packed size is fixed by (n, d, storage), except for block-sparse rows,
  // whose header (n, d, stored blocks) is read from the host copy.
  size_t want = 0;
  if (bcsr_storage(A->storage)) {
    NSRGS_CHECK_ARG(packed_bytes >= 64, "packed_bytes is smaller than the block-sparse header");
    const long long* hdr = static_cast<const long long*>(packed_host);
    NSRGS_CHECK_ARG(hdr[0] == n && hdr[1] == d && hdr[2] >= 0 && hdr[2] <= (long long)n * (n - 1),
                    "the block-sparse header does not match (n, d)");
    want = d <= 8 ? (size_t)bcsr_bytes(n, d, A->storage, hdr[2]) : 0;
  } else {
    want = nsrgs_packed_bytes(n, d, A->storage);
  }
  NSRGS_CHECK_ARG(want != 0, "unsupported (n, d, storage)");
  NSRGS_CHECK_ARG(packed_bytes == want, "packed_bytes differs from the packed size of (n, d, storage)");
  cudaStream_t st = (cudaStream_t)stv;
  const size_t xbytes = (size_t)n * d * d * sizeof(float);
  NSRGS_CUDA_TRY(cudaMemcpyAsync(const_cast<void*>(A->packed), packed_host, packed_bytes, cudaMemcpyHostToDevice, st));
  if (!init) {
    NSRGS_CHECK_ARG(X && aligned16(X), "X must be a 16-byte aligned device pointer");
    NSRGS_CUDA_TRY(cudaMemcpyAsync(X, X_host, xbytes, cudaMemcpyHostToDevice, st));
  }
  s = solve_impl(A, eta, T, K, tol, init, spectral_max_iters, X, info, ws, ws_bytes, stv, METHOD_NSRGS);
  if (s != NSRGS_OK) return s;
  NSRGS_CUDA_TRY(cudaMemcpyAsync(X_host, X, xbytes, cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
  return NSRGS_OK;
}

nsrgs_status nsrgs_objective(const nsrgs_A* A, const float* X, double* F, void* ws, size_t ws_bytes, void* stv) {
  PanelGeom g{};
  nsrgs_status s = check_A(A, &g);
  if (s != NSRGS_OK) return s;
  if ((s = check_ws(ws, ws_bytes, A->n, A->d)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(X && aligned16(X) && F, "X must be a 16-byte aligned device pointer and F non-null");
  const size_t bytes = (size_t)A->n * A->d * A->d * sizeof(float);
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, A->n, A->d);
  NSRGS_CUDA_TRY(maybe_tune(A, w, st));
  NSRGS_CUDA_TRY(reset_ws(w, A->n, A->d, st));
  NSRGS_CUDA_TRY(launch_norm2(A->packed, A->n, A->d, A->storage, g, w.obj, w.ctl, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(w.X[0], X, bytes, cudaMemcpyDeviceToDevice, st));
  NSRGS_CUDA_TRY(stream_AX(A, g, w.X[0], w, &w.ctl->stop, st));
  NSRGS_CUDA_TRY(launch_objective(w.X[0], w.Y, w.X[1], w.obj.Yprev, A->n, A->d, 0.0, w.obj, w.ctl, st));
  double oscal[OBJ_NSCAL];
  Ctl c{};
  NSRGS_CUDA_TRY(cudaMemcpyAsync(oscal, w.obj.scal, sizeof(oscal), cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaMemcpyAsync(&c, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
  if (c.flags & FLAG_BAD_LAYOUT) {
    set_error("the packed A is inconsistent: an index or address left its buffer (access skipped)");
    return NSRGS_ERR_INVALID_ARG;
  }
  if (c.flags & FLAG_TIMEOUT) {
    set_error("a device-side wait timed out");
    return NSRGS_ERR_TIMEOUT;
  }
  *F = oscal[OBJ_F];
  return NSRGS_OK;
}

static nsrgs_status solve_impl(const nsrgs_A* A, float eta, int T, int K, double tol, int init,
                               int spectral_max_iters, float* X, nsrgs_info* info, void* ws, size_t ws_bytes,
                               void* stv, int method, int safeguard) {
  PanelGeom g{};
  nsrgs_status s = check_A(A, &g);
  if (s != NSRGS_OK) return s;
  if ((s = check_small_d(A->d)) != NSRGS_OK) return s;
  if ((s = check_ws(ws, ws_bytes, A->n, A->d)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(eta > 0.f && isfinite(eta), "eta must be finite and > 0");
  NSRGS_CHECK_ARG(K >= 0 && K <= 64, "K must be in [0, 64]");
  NSRGS_CHECK_ARG(T >= 0 && T <= 100000, "T must be in [0, 100000]");
  NSRGS_CHECK_ARG((method == METHOD_NSRGS_OBJECTIVE || tol >= 0.0) && isfinite(tol), "tol must be finite and >= 0");
  NSRGS_CHECK_ARG(!init || (spectral_max_iters >= 1 && spectral_max_iters <= 10000),
                  "spectral_max_iters must be in [1, 10000]");
  NSRGS_CHECK_ARG(X && aligned16(X), "X must be a 16-byte aligned device pointer");
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, A->n, A->d);
  const int n = A->n, d = A->d;
  const size_t bytes = (size_t)n * d * d * sizeof(float);

  int dev = 0;
  NSRGS_CUDA_TRY(cudaGetDevice(&dev));
  GraphKey key;
  memset(&key, 0, sizeof(key));
  key.dev = dev;
  key.packed = A->packed;
  key.n = n;
  key.d = d;
  key.storage = A->storage;
  key.eta = eta;
  key.T = T;
  key.K = K;
  key.tol = tol;
  key.init = init ? 1 : 0;
  key.smax = init ? spectral_max_iters : 0;
  key.X = X;
  key.ws = ws;
  key.timing = g_timing;
  key.method = method;
  key.safeguard = safeguard ? 1 : 0;

  cudaGraphExec_t exec = nullptr;
  int kernel_nodes = 0;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (size_t k = 0; k < g_graphs.size(); ++k)
      if (g_graphs[k].key == key) {
        exec = g_graphs[k].exec;
        kernel_nodes = g_graphs[k].kernel_nodes;
        GraphEntry e = g_graphs[k];
        g_graphs.erase(g_graphs.begin() + k);
        g_graphs.push_back(e);
        break;
      }
  }
  if (!exec) {
    cudaStream_t cs;
    NSRGS_CUDA_TRY(capture_stream(dev, &cs));
    if (key.timing) NSRGS_CUDA_TRY(ensure_events(dev, T));
    const cudaEvent_t* ev = key.timing ? g_timing_state[dev].ev.data() : nullptr;
    // tuning and kernel attributes happen outside of capture
    NSRGS_CUDA_TRY(maybe_tune(A, w, st));
    NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
    NSRGS_CUDA_TRY(cudaStreamSynchronize(cs));
    NSRGS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = reset_ws(w, n, d, cs);
    if (e == cudaSuccess && method == METHOD_NSRGS_OBJECTIVE) e = launch_norm2(A->packed, n, d, A->storage, g, w.obj, w.ctl, cs);
    if (e == cudaSuccess) {
      if (init) e = enqueue_spectral(A, g, w, spectral_max_iters, 1e-6, w.X[0], cs);
      else e = cudaMemcpyAsync(w.X[0], X, bytes, cudaMemcpyDeviceToDevice, cs);
    }
    if (e == cudaSuccess) e = enqueue_iterations(A, g, w, eta, T, K, tol, method, key.safeguard, cs, ev);
    if (e == cudaSuccess) e = launch_copy_out(w.X[0], w.X[1], X, (long long)n * d * d, w.ctl, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      set_error(std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
      return NSRGS_ERR_CUDA;
    }
    kernel_nodes = count_kernel_nodes(graph);
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      return NSRGS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graphs.push_back(GraphEntry{key, exec, kernel_nodes});
    if (g_graphs.size() > 8) {
      cudaGraphExecDestroy(g_graphs.front().exec);
      g_graphs.erase(g_graphs.begin());
    }
  }
  NSRGS_CUDA_TRY(cudaGraphLaunch(exec, st));
  const bool looped = fused_loop(A, method) && T > 0;
  g_timing_state[dev].last_T = key.timing ? (looped ? 1 : T) : 0;
  g_timing_state[dev].per_pair = looped ? T : 1;
  g_timing_state[dev].last_nodes = kernel_nodes;
  if (info) {
    Ctl c{};
    double oscal[OBJ_NSCAL] = {};
    NSRGS_CUDA_TRY(cudaMemcpyAsync(&c, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    if (method == METHOD_NSRGS_OBJECTIVE)
      NSRGS_CUDA_TRY(cudaMemcpyAsync(oscal, w.obj.scal, sizeof(oscal), cudaMemcpyDeviceToHost, st));
    NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
    info->objective = (method == METHOD_NSRGS_OBJECTIVE && oscal[OBJ_EVALS] >= 1.0) ? oscal[OBJ_F] : NAN;
    info->rel_decrease = (method == METHOD_NSRGS_OBJECTIVE && oscal[OBJ_EVALS] >= 2.0) ? oscal[OBJ_R] : NAN;
    info->spectral_iters = c.spec_iters;
    info->iters = c.iters_done;
    info->last_update_norm = c.last_upd;
    info->spectral_residual = c.spec_res;
    info->flags = (c.flags & (FLAG_NONFINITE | FLAG_NS_PRECOND | FLAG_NS_SAFEGUARDED | FLAG_SPEC_SHIFTED |
                             FLAG_SPEC_AT_FLOOR)) |
                  ((init && !c.spec_stop) ? FLAG_SPEC_NOT_CONVERGED : 0);
    if (c.flags & FLAG_BAD_LAYOUT) {
      set_error("the packed A is inconsistent: an index or address left its buffer (access skipped)");
      return NSRGS_ERR_INVALID_ARG;
    }
    if (c.flags & FLAG_TIMEOUT) {
      set_error("a device-side wait timed out");
      return NSRGS_ERR_TIMEOUT;
    }
    if (c.flags & FLAG_NONFINITE) {
      set_error("an iterate became non-finite");
      return NSRGS_ERR_NONFINITE;
    }
  }
  return NSRGS_OK;
}

// ------------------------------------------------------------ SE(d) form
// FP8 is left out: its per-row scale stores the unit pair weights w_ij only to
// within ~6% of 1, which skews the translation Laplacian (measured: +4.5% on the
// translation error at n = 400 against the oracle, BF16 +0.1%).
static bool se_storage(int storage) { return storage == NSRGS_F32 || storage == NSRGS_BF16; }

size_t nsrgs_se_packed_bytes(int n, int d, int storage) {
  if (d < 1 || d > 63 || !se_storage(storage)) return 0;
  return nsrgs_packed_bytes(n, d + 1, storage);
}

size_t nsrgs_se_workspace_bytes(int n, int d) {
  if (d < 1 || d > 63) return 0;
  return nsrgs_workspace_bytes(n, d + 1);
}

nsrgs_status nsrgs_se_pack(const float* upper_a, const float* upper_c, int n, int d, float kappa, int storage,
                           void* packed, void* stv) {
  nsrgs_status s = check_nd(n, d);
  if (s != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(d <= 63, "the SE(d) form covers d <= 63 (augmented blocks of d + 1 <= 64)");
  NSRGS_CHECK_ARG(se_storage(storage), "the SE(d) form stores NSRGS_F32 or NSRGS_BF16");
  NSRGS_CHECK_ARG(kappa >= 0.f && isfinite(kappa), "kappa must be finite and >= 0");
  NSRGS_CHECK_ARG(upper_a && upper_c && packed && aligned16(packed), "null or misaligned pointer");
  return pack_se_impl(upper_a, upper_c, n, d, kappa, storage, packed, (cudaStream_t)stv);
}

nsrgs_status nsrgs_se_solve(const nsrgs_A* B, float kappa, float eta, float eta_t, int T, int K, double tol,
                            float* X, float* t, nsrgs_info* info, void* ws, size_t ws_bytes, void* stv) {
  NSRGS_CHECK_ARG(B != nullptr, "B is null");
  NSRGS_CHECK_ARG(B->d >= 2 && B->d <= 64 && se_storage(B->storage),
                  "B must be an nsrgs_se_pack result: d + 1 in [2, 64], NSRGS_F32 or NSRGS_BF16");
  PanelGeom g{};
  nsrgs_status s = check_A(B, &g);
  if (s != NSRGS_OK) return s;
  const int n = B->n, D = B->d, d = D - 1;
  if ((s = check_ws(ws, ws_bytes, n, D)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(kappa >= 0.f && isfinite(kappa), "kappa must be finite and >= 0");
  NSRGS_CHECK_ARG(eta > 0.f && isfinite(eta), "eta must be finite and > 0");
  NSRGS_CHECK_ARG(eta_t >= 0.f && isfinite(eta_t), "eta_t must be finite and >= 0");
  NSRGS_CHECK_ARG(K >= 0 && K <= 64, "K must be in [0, 64]");
  NSRGS_CHECK_ARG(T >= 0 && T <= 100000, "T must be in [0, 100000]");
  NSRGS_CHECK_ARG(tol >= 0.0 && isfinite(tol), "tol must be finite and >= 0");
  NSRGS_CHECK_ARG(X && t && aligned16(X) && aligned16(t), "X and t must be 16-byte aligned device pointers");
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, n, D);
  int dev = 0;
  NSRGS_CUDA_TRY(cudaGetDevice(&dev));
  const bool timing = g_timing != 0;
  if (timing) NSRGS_CUDA_TRY(ensure_events(dev, T));
  const cudaEvent_t* ev = timing ? g_timing_state[dev].ev.data() : nullptr;
  NSRGS_CUDA_TRY(se_prepare(d));
  NSRGS_CUDA_TRY(reset_ws(w, n, D, st));
  NSRGS_CUDA_TRY(se_launch(0, d, X, t, nullptr, nullptr, w.X[0], n, eta, eta_t, kappa, K, tol, w.ctl, nullptr, st));
  for (int it = 0; it < T; ++it) {
    if (ev) NSRGS_CUDA_TRY(cudaEventRecord(ev[2 * it], st));
    NSRGS_CUDA_TRY(stream_AX(B, g, w.X[it & 1], w, &w.ctl->stop, st));
    if (ev) NSRGS_CUDA_TRY(cudaEventRecord(ev[2 * it + 1], st));
    NSRGS_CUDA_TRY(se_launch(1, d, nullptr, t, w.X[it & 1], w.Y, w.X[(it + 1) & 1], n, eta, eta_t, kappa, K, tol,
                             w.ctl, nullptr, st));
  }
  NSRGS_CUDA_TRY(se_launch(2, d, nullptr, nullptr, w.X[0], nullptr, w.X[1], n, eta, eta_t, kappa, K, tol, w.ctl, X,
                           st));
  g_timing_state[dev].last_T = timing ? T : 0;
  g_timing_state[dev].per_pair = 1;
  g_timing_state[dev].last_nodes = 2 * T + 2;
  Ctl c{};
  NSRGS_CUDA_TRY(cudaMemcpyAsync(&c, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = c.iters_done;
    info->last_update_norm = c.last_upd;
    info->flags = c.flags & (FLAG_NONFINITE | FLAG_NS_PRECOND);
    info->objective = NAN;
    info->rel_decrease = NAN;
  }
  if (c.flags & FLAG_BAD_LAYOUT) {
    set_error("the packed matrix is inconsistent: an index or address left its buffer (access skipped)");
    return NSRGS_ERR_INVALID_ARG;
  }
  if (c.flags & FLAG_TIMEOUT) {
    set_error("a device-side wait timed out");
    return NSRGS_ERR_TIMEOUT;
  }
  if (c.flags & FLAG_NONFINITE) {
    set_error("an iterate became non-finite");
    return NSRGS_ERR_NONFINITE;
  }
  return NSRGS_OK;
}

nsrgs_status nsrgs_set_kernel_timing(int enable) {
  g_timing = enable ? 1 : 0;
  return NSRGS_OK;
}

nsrgs_status nsrgs_kernel_timing(int* launches, double* mean_ms, int* graph_kernel_nodes) {
  NSRGS_CHECK_ARG(launches && mean_ms, "launches and mean_ms must be non-null");
  int dev = 0;
  NSRGS_CUDA_TRY(cudaGetDevice(&dev));
  NSRGS_CUDA_TRY(cudaDeviceSynchronize());
  TimingState& ts = g_timing_state[dev];
  double sum = 0.0;
  for (int t = 0; t < ts.last_T; ++t) {
    float ms = 0.f;
    NSRGS_CUDA_TRY(cudaEventElapsedTime(&ms, ts.ev[2 * t], ts.ev[2 * t + 1]));
    sum += ms;
  }
  // per A pass: a timed pair covers per_pair iterations (the fused loop) or one
  *launches = ts.last_T * ts.per_pair;
  *mean_ms = ts.last_T ? sum / ts.last_T / ts.per_pair : 0.0;
  if (graph_kernel_nodes) *graph_kernel_nodes = ts.last_nodes;
  return NSRGS_OK;
}

nsrgs_status nsrgs_dF(const float* X, const float* Y, int n, int d, double* out, void* ws, size_t ws_bytes,
                      void* stv) {
  nsrgs_status s = check_nd(n, d);
  if (s != NSRGS_OK) return s;
  if ((s = check_small_d(d)) != NSRGS_OK) return s;
  if ((s = check_ws(ws, ws_bytes, n, d)) != NSRGS_OK) return s;
  NSRGS_CHECK_ARG(X && Y && out && aligned16(X) && aligned16(Y), "X, Y must be 16-byte aligned; out non-null");
  cudaStream_t st = (cudaStream_t)stv;
  Workspace w = map_workspace(ws, n, d);
  NSRGS_CUDA_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st));
  NSRGS_CUDA_TRY(launch_dF(X, Y, (long long)n * d, d, w.s, w.ctl, st));
  double r = 0.0;
  NSRGS_CUDA_TRY(cudaMemcpyAsync(&r, w.s.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  NSRGS_CUDA_TRY(cudaStreamSynchronize(st));
  *out = sqrt(r);
  return NSRGS_OK;
}

}  // extern "C"

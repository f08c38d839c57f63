// Serving form: continuous batching of NS-RGS solves.
//
// A server owns a fixed number of slots and sub-allocates a device arena that
// the caller provides (so admission is by HBM budget: a request is admitted
// when a slot is free and its packed A plus its scratch fit in the arena).
// Each nsrgs_server_step call
//   1. admits queued requests in arrival order (packs A into the arena, fills
//      the slot's instance entry, marks it PHASE_ADMIT),
//   2. replays one CUDA graph: the admit kernel, `ticks_per_step` ticks of the
//      batched form (one A-stream launch over every active slot + one phase
//      launch), and a report kernel,
//   3. reads the report and retires every slot whose request finished
//      (update norm below its tolerance, iteration cap, or a non-finite
//      iterate), freeing its arena space.
// Requests admitted while others run share the next ticks with them; each
// instance's arithmetic does not depend on who else is in the tick.
#include <string.h>

#include <algorithm>
#include <deque>
#include <string>
#include <vector>

#include "batch.cuh"

namespace nsrgs {
nsrgs_status pack_upper_impl(const float*, int, int, int, void*, cudaStream_t);
long long bcsr_bytes(int n, int d, int storage, long long nnzb);
}

using namespace nsrgs;

namespace {

// First-fit allocator over [begin, end) of the arena, 256-byte granules.
class RangeAlloc {
 public:
  void reset(size_t begin, size_t end) {
    free_.clear();
    if (end > begin) free_.push_back({begin, end - begin});
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (size_t k = 0; k < free_.size(); ++k) {
      if (free_[k].size >= bytes) {
        *off = free_[k].off;
        free_[k].off += bytes;
        free_[k].size -= bytes;
        if (free_[k].size == 0) free_.erase(free_.begin() + k);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = std::lower_bound(free_.begin(), free_.end(), off,
                               [](const Range& r, size_t o) { return r.off < o; });
    it = free_.insert(it, {off, bytes});
    // coalesce with neighbours
    size_t k = it - free_.begin();
    if (k + 1 < free_.size() && free_[k].off + free_[k].size == free_[k + 1].off) {
      free_[k].size += free_[k + 1].size;
      free_.erase(free_.begin() + k + 1);
    }
    if (k > 0 && free_[k - 1].off + free_[k - 1].size == free_[k].off) {
      free_[k - 1].size += free_[k].size;
      free_.erase(free_.begin() + k);
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (const Range& r : free_) m = std::max(m, r.size);
    return m;
  }

 private:
  struct Range {
    size_t off, size;
  };
  std::vector<Range> free_;
};

struct Request {
  uint64_t id;
  const float* upper;
  int n;
  float eta;
  int Tmax;
  double tol;
  float* X;
  int sparse;          // 1: block-sparse rows
  size_t packed_bytes;  // exact packed size of a block-sparse request
};

struct Slot {
  bool busy = false;
  uint64_t id = 0;
  size_t a_off = 0, a_bytes = 0, w_off = 0, w_bytes = 0;
};

const int kAdmitPhase = PHASE_ADMIT;

}  // namespace

struct nsrgs_server {
  nsrgs_server_config cfg;
  uint8_t* arena = nullptr;
  size_t arena_bytes = 0;
  cudaStream_t st = nullptr;
  BatchDesc* d_descs = nullptr;
  long long* d_base = nullptr;
  long long* d_rbase = nullptr;  // first global row of each slot's block-sparse rows
  long long* d_bbase = nullptr;  // first global block of each slot
  int* d_nspec = nullptr;        // slots in a spectral phase
  BatchReport* d_rep = nullptr;
  std::vector<BatchDesc> h_descs;
  std::vector<Ctl*> idle_ctl;  // per slot: zeroed control block used while the slot is free
  std::vector<long long> h_base, h_rbase, h_bbase;
  std::vector<BatchReport> h_rep;
  std::vector<Slot> slots;
  std::deque<Request> queue;
  std::vector<nsrgs_server_result> finished;
  RangeAlloc alloc;
  cudaGraphExec_t exec = nullptr;
  uint64_t next_id = 1;
  bool dirty = true;
};

static size_t server_table_bytes(int max_slots) { return batch_table_bytes(max_slots); }

extern "C" size_t nsrgs_server_table_bytes(int max_slots) {
  if (max_slots < 1) return 0;
  return server_table_bytes(max_slots);
}

extern "C" nsrgs_status nsrgs_server_create(const nsrgs_server_config* cfg, void* arena, size_t arena_bytes, void* st,
                                            nsrgs_server** out) {
  NSRGS_CHECK_ARG(cfg && out, "cfg and out must be non-null");
  NSRGS_CHECK_ARG(cfg->d >= 1 && cfg->d <= 4, "the served form covers 1 <= d <= 4");
  NSRGS_CHECK_ARG(cfg->storage >= NSRGS_F32 && cfg->storage <= NSRGS_FP8E4M3, "storage must be F32, BF16 or FP8E4M3");
  NSRGS_CHECK_ARG(cfg->max_slots >= 1 && cfg->max_slots <= 65536, "max_slots in [1, 65536]");
  NSRGS_CHECK_ARG(cfg->K >= 0 && cfg->K <= 64, "K in [0, 64]");
  NSRGS_CHECK_ARG(cfg->spectral_max_iters >= 1 && cfg->spectral_max_iters <= 10000, "spectral_max_iters in [1, 10000]");
  NSRGS_CHECK_ARG(cfg->ticks_per_step >= 1 && cfg->ticks_per_step <= 4096, "ticks_per_step in [1, 4096]");
  NSRGS_CHECK_ARG(cfg->spectral_tol >= 0.0, "spectral_tol >= 0");
  NSRGS_CHECK_ARG(arena && (reinterpret_cast<uintptr_t>(arena) & 255u) == 0, "arena must be 256-byte aligned");
  const size_t tb = server_table_bytes(cfg->max_slots);
  if (arena_bytes < tb) {
    set_error("arena smaller than nsrgs_server_table_bytes(max_slots)");
    return NSRGS_ERR_NOMEM;
  }
  nsrgs_server* s = new nsrgs_server();
  s->cfg = *cfg;
  s->arena = reinterpret_cast<uint8_t*>(arena);
  s->arena_bytes = arena_bytes;
  s->st = (cudaStream_t)st;
  const int M = cfg->max_slots;
  const size_t tbytes = ((size_t)M * sizeof(BatchDesc) + 255) / 256 * 256;
  const size_t bbytes = ((size_t)(M + 1) * sizeof(long long) + 255) / 256 * 256;
  s->d_descs = reinterpret_cast<BatchDesc*>(s->arena);
  s->d_base = reinterpret_cast<long long*>(s->arena + tbytes);
  s->d_rep = reinterpret_cast<BatchReport*>(s->arena + tbytes + bbytes);
  const size_t rbytes = ((size_t)M * sizeof(BatchReport) + 255) / 256 * 256;
  s->d_rbase = reinterpret_cast<long long*>(s->arena + tbytes + bbytes + rbytes);
  s->d_bbase = reinterpret_cast<long long*>(s->arena + tbytes + 2 * bbytes + rbytes);
  s->d_nspec = reinterpret_cast<int*>(s->arena + tbytes + 3 * bbytes + rbytes);
  s->h_descs.assign(M, BatchDesc{});
  s->h_base.assign(M + 1, 0);
  s->h_rbase.assign(M + 1, 0);
  s->h_bbase.assign(M + 1, 0);
  s->h_rep.assign(M, BatchReport{});
  s->slots.assign(M, Slot{});
  s->alloc.reset(tb, arena_bytes);
  // Idle entries point at a private scratch-free dummy: their control blocks
  // live in a small shared area so kernels can read phase == PHASE_IDLE.
  size_t ctl_off = 0;
  if (!s->alloc.alloc(256 * (size_t)M, &ctl_off)) {
    delete s;
    set_error("arena too small for the slot control blocks");
    return NSRGS_ERR_NOMEM;
  }
  s->idle_ctl.assign(M, nullptr);
  for (int i = 0; i < M; ++i) {
    memset(&s->h_descs[i], 0, sizeof(BatchDesc));
    s->idle_ctl[i] = reinterpret_cast<Ctl*>(s->arena + ctl_off + 256 * (size_t)i);
    s->h_descs[i].ctl = s->idle_ctl[i];
  }
  cudaError_t e = cudaMemsetAsync(s->arena + ctl_off, 0, 256 * (size_t)M, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_nspec, 0, sizeof(int), s->st);
  if (e == cudaSuccess) e = batch_stream(nullptr, nullptr, 0, cfg->d, cfg->storage, s->st, true);
  if (e != cudaSuccess) {
    delete s;
    set_error(std::string("server set-up: ") + cudaGetErrorString(e));
    return NSRGS_ERR_CUDA;
  }
  *out = s;
  return NSRGS_OK;
}

// Block-sparse requests take the element type of the server's panel storage.
static int sparse_storage(const nsrgs_server* s) { return s->cfg.storage == NSRGS_F32 ? NSRGS_BCSR_F32 : NSRGS_BCSR_BF16; }

extern "C" nsrgs_status nsrgs_server_submit(nsrgs_server* s, const float* upper, int n, float eta, int T_max,
                                            double tol, float* X, uint64_t* id) {
  return nsrgs_server_submit_ex(s, upper, n, eta, T_max, tol, 0, 0, X, id);
}

extern "C" nsrgs_status nsrgs_server_submit_ex(nsrgs_server* s, const float* upper, int n, float eta, int T_max,
                                               double tol, int sparse, size_t packed_bytes, float* X, uint64_t* id) {
  NSRGS_CHECK_ARG(s && upper && X && id, "null argument");
  NSRGS_CHECK_ARG(n >= 2, "n must be >= 2");
  NSRGS_CHECK_ARG(!sparse || packed_bytes >= (size_t)bcsr_bytes(n, s->cfg.d, sparse_storage(s), 0),
                  "a block-sparse request needs its packed size (nsrgs_bcsr_packed_bytes)");
  NSRGS_CHECK_ARG(n >= 2 && (long long)n * s->cfg.d <= (1LL << 24), "n out of range");
  NSRGS_CHECK_ARG(eta > 0.f && isfinite(eta), "eta must be finite and > 0");
  NSRGS_CHECK_ARG(T_max >= 1 && T_max <= 1000000, "T_max in [1, 1000000]");
  NSRGS_CHECK_ARG(tol >= 0.0 && isfinite(tol), "tol must be finite and >= 0");
  NSRGS_CHECK_ARG((reinterpret_cast<uintptr_t>(X) & 15u) == 0, "X must be 16-byte aligned");
  const size_t abytes = sparse ? packed_bytes : nsrgs_packed_bytes(n, s->cfg.d, s->cfg.storage);
  const size_t need = abytes + batch_instance_bytes(n, s->cfg.d) + 512;
  if (need > s->arena_bytes - server_table_bytes(s->cfg.max_slots)) {
    set_error("request can never fit in the server's arena");
    return NSRGS_ERR_NOMEM;
  }
  Request r{s->next_id++, upper, n, eta, T_max, tol, X, sparse ? 1 : 0, abytes};
  s->queue.push_back(r);
  *id = r.id;
  return NSRGS_OK;
}

static cudaError_t server_capture(nsrgs_server* s) {
  const int M = s->cfg.max_slots, d = s->cfg.d;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = batch_admit(s->d_descs, M, d, s->d_nspec, cs);
    for (int t = 0; t < s->cfg.ticks_per_step && e == cudaSuccess; ++t) {
      e = batch_stream(s->d_descs, s->d_base, M, d, s->cfg.storage, cs, false);
      // block-sparse slots (none: the row kernel finds no rows and returns)
      if (e == cudaSuccess)
        e = batch_bcsr_stream(s->d_descs, s->d_rbase, M, d, sparse_storage(s) == NSRGS_BCSR_BF16, 1LL << 40, cs);
      if (e == cudaSuccess) e = batch_spec(s->d_descs, s->d_bbase, M, d, 1LL << 40, s->d_nspec, cs);
      // grid sized for a full table; blocks past the current total return at once
      if (e == cudaSuccess) e = batch_block(s->d_descs, s->d_bbase, M, d, 1LL << 40, cs);
    }
    if (e == cudaSuccess) e = batch_report(s->d_descs, M, s->d_rep, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
  }
  cudaStreamDestroy(cs);
  return e;
}

extern "C" nsrgs_status nsrgs_server_step(nsrgs_server* s, int* active, int* queued) {
  NSRGS_CHECK_ARG(s != nullptr, "server is null");
  const int M = s->cfg.max_slots, d = s->cfg.d, storage = s->cfg.storage;
  // 1. admission by slot and arena space, in arrival order
  while (!s->queue.empty()) {
    int free_slot = -1;
    for (int i = 0; i < M; ++i)
      if (!s->slots[i].busy) {
        free_slot = i;
        break;
      }
    if (free_slot < 0) break;
    const Request& r = s->queue.front();
    const int rstorage = r.sparse ? sparse_storage(s) : storage;
    const size_t abytes = r.packed_bytes;
    const size_t wbytes = batch_instance_bytes(r.n, d);
    size_t aoff = 0, woff = 0;
    if (!s->alloc.alloc(abytes, &aoff)) break;
    if (!s->alloc.alloc(wbytes, &woff)) {
      s->alloc.release(aoff, abytes);
      break;
    }
    nsrgs_status ps = pack_upper_impl(r.upper, r.n, d, rstorage, s->arena + aoff, s->st);
    if (ps != NSRGS_OK) return ps;
    Slot& sl = s->slots[free_slot];
    sl.busy = true;
    sl.id = r.id;
    sl.a_off = aoff;
    sl.a_bytes = abytes;
    sl.w_off = woff;
    sl.w_bytes = wbytes;
    BatchDesc& ds = s->h_descs[free_slot];
    memset(&ds, 0, sizeof(ds));
    if (r.sparse) {
      ds.sparse = 1;  // no panel steps: streamed by the row kernel
      ds.g.n = r.n;
      ds.g.D = d;
      ds.g.storage = rstorage;
    } else {
      make_panel_geom(r.n, d, storage, &ds.g);
    }
    ds.packed = s->arena + aoff;
    fill_instance(ds, s->arena + woff, r.n, d);
    ds.Xout = r.X;
    ds.eta = r.eta;
    ds.T = r.Tmax;
    ds.K = s->cfg.K;
    ds.smax = s->cfg.spectral_max_iters;
    ds.start_given = 0;
    ds.safeguard = s->cfg.ns_safeguard ? 1 : 0;
    ds.tol = r.tol;
    ds.spec_tol = s->cfg.spectral_tol;
    NSRGS_CUDA_TRY(cudaMemcpyAsync(&ds.ctl->phase, &kAdmitPhase, sizeof(int), cudaMemcpyHostToDevice, s->st));
    s->queue.pop_front();
    s->dirty = true;
  }
  // 2. instance table: only busy slots contribute steps (even split over active work)
  if (s->dirty) {
    long long steps = 0, rows = 0, blocks = 0;
    for (int i = 0; i < M; ++i) {
      s->h_base[i] = steps;
      s->h_rbase[i] = rows;
      s->h_bbase[i] = blocks;
      if (s->slots[i].busy) {
        steps += s->h_descs[i].g.total_steps;
        if (s->h_descs[i].sparse) rows += s->h_descs[i].g.n;
        blocks += s->h_descs[i].g.n;
      }
    }
    s->h_base[M] = steps;
    s->h_rbase[M] = rows;
    s->h_bbase[M] = blocks;
    NSRGS_CUDA_TRY(cudaMemcpyAsync(s->d_rbase, s->h_rbase.data(), sizeof(long long) * (M + 1),
                                   cudaMemcpyHostToDevice, s->st));
    NSRGS_CUDA_TRY(cudaMemcpyAsync(s->d_bbase, s->h_bbase.data(), sizeof(long long) * (M + 1),
                                   cudaMemcpyHostToDevice, s->st));
    NSRGS_CUDA_TRY(cudaMemcpyAsync(s->d_descs, s->h_descs.data(), sizeof(BatchDesc) * M, cudaMemcpyHostToDevice, s->st));
    NSRGS_CUDA_TRY(cudaMemcpyAsync(s->d_base, s->h_base.data(), sizeof(long long) * (M + 1), cudaMemcpyHostToDevice,
                                   s->st));
    s->dirty = false;
  }
  if (!s->exec) NSRGS_CUDA_TRY(server_capture(s));
  int busy = 0;
  for (int i = 0; i < M; ++i) busy += s->slots[i].busy ? 1 : 0;
  if (busy > 0) {
    // 3. ticks, then retire finished requests
    NSRGS_CUDA_TRY(cudaGraphLaunch(s->exec, s->st));
    NSRGS_CUDA_TRY(cudaMemcpyAsync(s->h_rep.data(), s->d_rep, sizeof(BatchReport) * M, cudaMemcpyDeviceToHost, s->st));
    NSRGS_CUDA_TRY(cudaStreamSynchronize(s->st));
    for (int i = 0; i < M; ++i) {
      Slot& sl = s->slots[i];
      if (!sl.busy || s->h_rep[i].phase != PHASE_DONE) continue;
      const BatchReport& r = s->h_rep[i];
      nsrgs_server_result res;
      res.id = sl.id;
      res.status = (r.flags & FLAG_BAD_LAYOUT) ? NSRGS_ERR_INVALID_ARG
                   : (r.flags & FLAG_TIMEOUT)  ? NSRGS_ERR_TIMEOUT
                   : (r.flags & FLAG_NONFINITE) ? NSRGS_ERR_NONFINITE
                                                : NSRGS_OK;
      res.iters = r.iters;
      res.spectral_iters = r.spec_iters;
      res.last_update_norm = r.last_upd;
      res.flags = r.flags & (FLAG_NONFINITE | FLAG_NS_PRECOND | FLAG_SPEC_SHIFTED);
      s->finished.push_back(res);
      s->alloc.release(sl.a_off, sl.a_bytes);
      s->alloc.release(sl.w_off, sl.w_bytes);
      // the freed arena space may be reused at once: point the entry back at
      // the slot's idle control block (phase PHASE_IDLE) before the next tick
      memset(&s->h_descs[i], 0, sizeof(BatchDesc));
      s->h_descs[i].ctl = s->idle_ctl[i];
      sl.busy = false;
      s->dirty = true;
      busy -= 1;
    }
  }
  if (active) *active = busy;
  if (queued) *queued = (int)s->queue.size();
  return NSRGS_OK;
}

extern "C" nsrgs_status nsrgs_server_poll(nsrgs_server* s, nsrgs_server_result* out, int max, int* count) {
  NSRGS_CHECK_ARG(s && count && (out || max == 0), "null argument");
  const int k = std::min<int>(max, (int)s->finished.size());
  for (int i = 0; i < k; ++i) out[i] = s->finished[i];
  s->finished.erase(s->finished.begin(), s->finished.begin() + k);
  *count = k;
  return NSRGS_OK;
}

extern "C" void nsrgs_server_destroy(nsrgs_server* s) {
  if (!s) return;
  if (s->exec) cudaGraphExecDestroy(s->exec);
  delete s;
}

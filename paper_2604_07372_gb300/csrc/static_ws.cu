// nsrgs_step_static: one NS-RGS iteration whose scratch lives in a fixed,
// file-scope device array instead of a caller-provided workspace.
//
// Who needs it: callers that cannot obtain device memory at the point where
// they run an iteration -- for example code embedded in a host program whose
// memory manager owns the whole device heap and hands out no scratch buffers,
// or a latency-critical loop that is not allowed to enter any allocator.
// Those callers still own X_in / X_out and the packed A; only the scratch
// moves into this library.
//
// Cost and limits: every GPU on which this entry point runs holds
// kStaticWorkspaceBytes (8 MiB) of device memory for this array until the
// process exits.  A problem whose workspace (nsrgs_workspace_bytes(n, d))
// exceeds that size is rejected with NSRGS_ERR_INVALID_ARG: the largest n is
// 418368 at d = 1, 46016 at d = 3, 25656 at d = 4, 6025 at d = 8 and 931 at
// d = 16; d >= 32 never fits (the float64 per-CTA partials alone exceed it).
// The array's device address is resolved once per device and cached, so the
// entry point must not be used across a cudaDeviceReset of that device (the
// module is reloaded and the cached address would be stale).
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticWorkspaceBytes = 8u << 20;

// The scratch itself.  Host code must not pass `g_static_workspace` to a kernel
// directly: on the host side the name is a stand-in, not a device address.
// The device address is fetched once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {};

}  // namespace

extern "C" nsrgs_status nsrgs_step_static(const nsrgs_A* A, float eta, int K, const float* X_in, float* X_out,
                                          double* upd_norm, void* st) {
  if (A == nullptr) {
    nsrgs::set_error("A is null");
    return NSRGS_ERR_INVALID_ARG;
  }
  const size_t need = nsrgs_workspace_bytes(A->n, A->d);
  if (need == 0) {
    nsrgs::set_error("n must be >= 2 and d in [1, 64]");
    return NSRGS_ERR_INVALID_ARG;
  }
  if (need > kStaticWorkspaceBytes) {
    nsrgs::set_error("nsrgs_step_static: this (n, d) needs " + std::to_string(need) +
                     " bytes of scratch, more than the fixed 8 MiB (8388608 bytes) array; use nsrgs_step "
                     "with a caller-provided workspace");
    return NSRGS_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    nsrgs::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return NSRGS_ERR_CUDA;
  }
  if (dev < 0 || dev >= 64) {
    nsrgs::set_error("nsrgs_step_static: device ordinal " + std::to_string(dev) +
                     " is not supported (the per-device address table holds ordinals 0..63)");
    return NSRGS_ERR_INVALID_ARG;
  }
  void* ptr = nullptr;
  {
    // One-time set-up per device, with that device current: resolve the
    // array's device address.
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
      e = cudaGetSymbolAddress(&g_static_ptr[dev], g_static_workspace);
      if (e != cudaSuccess) {
        g_static_ptr[dev] = nullptr;
        nsrgs::set_error(std::string("cudaGetSymbolAddress(static workspace): ") + cudaGetErrorString(e));
        return NSRGS_ERR_CUDA;
      }
    }
    ptr = g_static_ptr[dev];
  }
  // nsrgs_step clears everything that must start at zero (control block, Y
  // accumulator, X padding) before its kernels run, so leftovers of the
  // previous call in the shared array do not matter.
  return nsrgs_step(A, eta, K, X_in, X_out, upd_norm, ptr, kStaticWorkspaceBytes, st);
}

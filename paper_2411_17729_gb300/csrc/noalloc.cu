// noalloc.cu -- cascade_forward_fixed_scratch: the forward pass with its
// workspace taken from a fixed device array compiled into the library, for
// callers that cannot call cudaMalloc (see include/cascade.h).
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds CASCADE_FIXED_SCRATCH_BYTES of device memory until the
// process exits.  In host code its name is only a host-side stand-in: the
// device address is resolved once per device with cudaGetSymbolAddress and
// cached here.
#include "common.cuh"

#include <stdio.h>

#include <mutex>

namespace cascade {
cascade_status_t forward_with_workspace(Plan* p, const void* u, void* y, void* ws,
                                        cudaStream_t st);
size_t forward_workspace_bytes(const Plan& p);
}  // namespace cascade

using namespace cascade;

struct cascade_plan_s : public Plan {};

namespace {

static __device__ __align__(256) uint8_t g_fixed_scratch[CASCADE_FIXED_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

cascade_status_t nofail(Plan* p, cascade_status_t st, const std::string& msg) {
  if (p) p->last_error = msg;
  set_global_error(msg);
  return st;
}

// Device address of g_fixed_scratch on the current device (resolved once).
cascade_status_t scratch_on_current_device(Plan* p, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nofail(p, CASCADE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nofail(p, CASCADE_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    // With lazy module loading this first lookup loads the module that holds
    // the array, which commits its device memory now: an out-of-memory
    // failure there is reported as such.
    e = cudaGetSymbolAddress(&ptr, g_fixed_scratch);
    if (e != cudaSuccess || !ptr) {
      const cascade_status_t code =
          e == cudaErrorMemoryAllocation ? CASCADE_ERR_OOM : CASCADE_ERR_CUDA;
      if (e != cudaSuccess) cudaGetLastError();   // reset the runtime's last-error state
      return nofail(p, code,
                    std::string("cudaGetSymbolAddress(fixed scratch): ") + cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return CASCADE_OK;
}

}  // namespace

extern "C" cascade_status_t cascade_forward_fixed_scratch(cascade_plan_t plan, const void* d_u,
                                                          void* d_y, void* stream) {
  Plan* p = plan;
  if (!p) return nofail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!p->have_system || !p->have_batch)
    return nofail(p, CASCADE_ERR_STATE, "system and batch must be set");
  if (p->rows == 0) return CASCADE_OK;
  if (!d_u || !d_y) return nofail(p, CASCADE_ERR_INVALID_ARG, "u and y must be device pointers");
  if (!row_aligned(d_u) || !row_aligned(d_y))
    return nofail(p, CASCADE_ERR_INVALID_ARG, "u and y must be 16-byte aligned");
  if (p->timing)
    return nofail(p, CASCADE_ERR_UNSUPPORTED,
                  "disable stage timing first (it creates CUDA events)");
  if (p->device != -1) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != p->device)
      return nofail(p, CASCADE_ERR_INVALID_ARG, "the plan's device is not the current device");
  }
  const size_t need = forward_workspace_bytes(*p);
  if (need > (size_t)CASCADE_FIXED_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "batch needs %zu bytes of workspace; the fixed scratch holds %zu bytes "
             "(use cascade_forward with a caller-provided workspace)",
             need, (size_t)CASCADE_FIXED_SCRATCH_BYTES);
    return nofail(p, CASCADE_ERR_UNSUPPORTED, buf);
  }
  void* ws = nullptr;
  cascade_status_t r = scratch_on_current_device(p, &ws);
  if (r != CASCADE_OK) return r;
  // Every workspace byte the forward reads is written earlier in the same
  // call, so the previous call's contents need no clearing.  The stage
  // outputs a SAVE_STATES or RECOMPUTE plan keeps land in the shared array,
  // which the next call may overwrite: they are not offered to
  // cascade_backward, whose record of the last forward stays as it was.
  const void* const saved_ws = p->saved_ws;
  const int64_t saved_batch = p->saved_batch;
  const cascade_status_t r2 =
      forward_with_workspace(p, d_u, d_y, ws, static_cast<cudaStream_t>(stream));
  p->saved_ws = saved_ws;
  p->saved_batch = saved_batch;
  return r2;
}

// Allocation-free variant of fc_tx_synthesize.
//
// Who needs it: callers that must not allocate device memory while they run —
// for example a real-time radio loop whose memory budget is fixed before it
// starts, or a host process whose allocator is owned by another framework that
// the FC library cannot call into. fc_tx_synthesize asks such a caller for a
// workspace buffer (continuous mode keeps the low-rate CP-OFDM stream there);
// fc_tx_synthesize_static instead uses one file-scope device array, so the call
// itself allocates nothing.
//
// When the array is reserved: the library is built without relocatable device code,
// so this file is a CUDA module of its own, and with lazy module loading (the
// default since CUDA 12.2) the driver reserves the array only when the module is
// first touched. fc_plan_create therefore looks up the array's address on the plan's
// device (fc_internal_static_resolve), so the memory is taken at set-up, before any
// run-time call. Cost: every GPU on which a plan was created holds
// FC_STATIC_WORKSPACE_BYTES of device memory until the process exits, whether or not
// this entry point is used.
//
// The address is cached per device for the life of the process; a cudaDeviceReset
// (or a release and re-creation of the primary context) would leave it stale, so
// neither is supported while this library is in use.
#include <cstdio>
#include <mutex>

#include "fc_internal.cuh"
#include "fc_trace.h"

// One workspace shared by every call on a device (the contents of the last call stay there).
static __device__ __align__(256) unsigned char g_fc_static_workspace[FC_STATIC_WORKSPACE_BYTES];

namespace {

std::mutex g_static_mu;
void* g_static_ptr[64] = {};   // device address of the array, per device, resolved once

}  // namespace

int fc_internal_static_resolve(int dev) {
  if (dev < 0 || dev >= 64) return fc_internal_fail(FC_ERR_INVALID, "plan device out of range");
  // Look up the array's device address once per device, with that device current.
  // The host-side name of the array is only a stand-in and must never be handed to
  // a kernel.
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev]) return FC_OK;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fc_internal_fail(FC_ERR_CUDA, "cudaGetDevice failed");
  if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_fc_static_workspace);
  if (prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();   // an allocation failure here is not sticky; do not leave it for later launches
    if (e == cudaErrorMemoryAllocation)
      return fc_internal_fail(FC_ERR_NOMEM, "no device memory for the static workspace (loading its module)");
    return fc_internal_fail(FC_ERR_CUDA, "cudaGetSymbolAddress of the static workspace failed");
  }
  g_static_ptr[dev] = p;
  return FC_OK;
}

extern "C" int fc_tx_synthesize_static(const fc_plan* plan, int32_t n_streams, const void* grid_in, void* wave_out,
                                       void* stream) {
  FcRange nvtx_range(__func__);
  if (!plan) return fc_internal_fail(FC_ERR_INVALID, "plan is NULL");
  if (n_streams < 0) return fc_internal_fail(FC_ERR_INVALID, "n_streams < 0");
  fc_sizes sz;
  int rc = fc_query(plan, &sz);
  if (rc != FC_OK) return rc;
  const unsigned long long need = (unsigned long long)n_streams * (unsigned long long)sz.workspace_per_stream;
  if (need > FC_STATIC_WORKSPACE_BYTES) {
    char msg[160];
    snprintf(msg, sizeof msg, "static workspace too small: %llu bytes needed, %llu available (reduce n_streams)",
             need, (unsigned long long)FC_STATIC_WORKSPACE_BYTES);
    return fc_internal_fail(FC_ERR_INVALID, msg);
  }
  const int dev = fc_internal_plan_device(plan);
  // normally resolved already by fc_plan_create; resolved here if that attempt failed
  rc = fc_internal_static_resolve(dev);
  if (rc != FC_OK) return rc;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    ws = g_static_ptr[dev];
  }
  // Nothing in the workspace needs clearing: every element the TX kernels read
  // is written earlier in the same call.
  return fc_tx_synthesize(plan, n_streams, grid_in, wave_out, need ? ws : nullptr, need ? (size_t)need : 0, stream);
}

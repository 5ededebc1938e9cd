// Allocation-free variant of fc_tx_synthesize.
//
// Who needs it: callers that must not allocate device memory while they run —
// for example a real-time radio loop whose memory budget is fixed before it
// starts, or a host process whose allocator is owned by another framework that
// the FC library cannot call into. fc_tx_synthesize asks such a caller for a
// workspace buffer (continuous mode keeps the low-rate CP-OFDM stream there);
// fc_tx_synthesize_static instead uses one file-scope device array that is
// reserved when the library is loaded, so the call itself allocates nothing.
//
// Cost: every GPU that loads the library holds FC_STATIC_WORKSPACE_BYTES of
// device memory until the process exits, whether or not this entry point is used.
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
  if (dev < 0 || dev >= 64) return fc_internal_fail(FC_ERR_INVALID, "plan device out of range");
  void* ws = nullptr;
  {
    // First use on this device: look up the array's device address with that
    // device current. The host-side name of the array is only a stand-in and
    // must never be handed to a kernel.
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      int prev = -1;
      if (cudaGetDevice(&prev) != cudaSuccess) return fc_internal_fail(FC_ERR_CUDA, "cudaGetDevice failed");
      if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
        return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_fc_static_workspace);
      if (prev != dev) cudaSetDevice(prev);
      if (e != cudaSuccess || !p) return fc_internal_fail(FC_ERR_CUDA, "cudaGetSymbolAddress of the static workspace failed");
      g_static_ptr[dev] = p;
    }
    ws = g_static_ptr[dev];
  }
  // Nothing in the workspace needs clearing: every element the TX kernels read
  // is written earlier in the same call.
  return fc_tx_synthesize(plan, n_streams, grid_in, wave_out, need ? ws : nullptr, need ? (size_t)need : 0, stream);
}

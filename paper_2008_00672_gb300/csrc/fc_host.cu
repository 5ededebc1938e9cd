// Host-buffer execute calls: grids and waveforms in host memory, processed in chunks of
// streams whose host-to-device copy, FC kernels and device-to-host copy overlap across
// chunks (the copy engines of both directions and the SMs work at the same time).
//
// A pipeline owns `depth` slots of device buffers (input, output and workspace for
// `chunk_streams` streams) and one CUDA stream ("lane") per slot. Chunk i runs on lane
// i mod depth, so a slot is reused only after the lane has finished the chunk before it;
// the lanes fork from the caller's stream and join back into it.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fc_internal.cuh"
#include "fc_trace.h"

struct fc_pipeline {
  const fc_plan* plan = nullptr;
  int device = 0;
  int chunk = 0;
  fc_sizes sz{};
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  std::vector<unsigned char*> grid, wave;
  std::vector<void*> ws;
  size_t ws_bytes = 0;
  std::vector<void*> owned;
};

namespace {

struct DevGuard {
  int prev = -1;
  bool ok = false;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int cuda_err(cudaError_t e, const char* where) {
  char msg[200];
  snprintf(msg, sizeof msg, "%s: %s", where, cudaGetErrorString(e));
  return fc_internal_fail(e == cudaErrorMemoryAllocation ? FC_ERR_NOMEM : FC_ERR_CUDA, msg);
}

void release(fc_pipeline* p) {
  for (cudaEvent_t e : p->done) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  for (cudaStream_t s : p->lanes) cudaStreamDestroy(s);
  for (void* m : p->owned) cudaFree(m);
}

// direction FC_TX: host grid -> host wave; FC_RX: host wave -> host grid
int run(fc_pipeline* p, int dir, int32_t n_streams, const void* host_in, void* host_out, void* stream) {
  if (!p) return fc_internal_fail(FC_ERR_INVALID, "pipeline is NULL");
  if (n_streams < 0) return fc_internal_fail(FC_ERR_INVALID, "n_streams < 0");
  if (n_streams == 0) return FC_OK;
  if (!host_in || !host_out) return fc_internal_fail(FC_ERR_INVALID, "host buffer is NULL");
  DevGuard dg(p->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  const size_t in_len = (size_t)(dir == FC_TX ? p->sz.tx_in_len : p->sz.wave_len);
  const size_t out_len = (size_t)(dir == FC_TX ? p->sz.wave_len : p->sz.rx_out_len);
  const cudaStream_t caller = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(p->fork, caller);
  for (size_t l = 0; l < p->lanes.size() && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(p->lanes[l], p->fork, 0);
  if (e != cudaSuccess) return cuda_err(e, "pipeline fork");
  const int n_chunks = (n_streams + p->chunk - 1) / p->chunk;
  int used = 0;
  for (int c = 0; c < n_chunks; ++c) {
    const int slot = c % (int)p->lanes.size();
    used = std::max(used, slot + 1);
    const cudaStream_t st = p->lanes[slot];
    const int s0 = c * p->chunk, ns = std::min(p->chunk, n_streams - s0);
    const size_t sb = (size_t)p->sz.sample_bytes;   // complex64 or complex BF16
    unsigned char* d_in = dir == FC_TX ? p->grid[slot] : p->wave[slot];
    unsigned char* d_out = dir == FC_TX ? p->wave[slot] : p->grid[slot];
    e = cudaMemcpyAsync(d_in, (const unsigned char*)host_in + (size_t)s0 * in_len * sb, (size_t)ns * in_len * sb,
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_err(e, "pipeline host-to-device copy");
    const int rc = dir == FC_TX ? fc_tx_synthesize(p->plan, ns, d_in, d_out, p->ws[slot], p->ws_bytes, (void*)st)
                                : fc_rx_analyze(p->plan, ns, d_in, d_out, p->ws[slot], p->ws_bytes, (void*)st);
    if (rc != FC_OK) return rc;
    e = cudaMemcpyAsync((unsigned char*)host_out + (size_t)s0 * out_len * sb, d_out, (size_t)ns * out_len * sb,
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_err(e, "pipeline device-to-host copy");
  }
  for (int l = 0; l < used && e == cudaSuccess; ++l) {
    e = cudaEventRecord(p->done[l], p->lanes[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, p->done[l], 0);
  }
  return e == cudaSuccess ? FC_OK : cuda_err(e, "pipeline join");
}

}  // namespace

extern "C" {

int fc_pipeline_create(const fc_plan* plan, int32_t chunk_streams, int32_t depth, fc_pipeline** out) {
  if (!out) return fc_internal_fail(FC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!plan) return fc_internal_fail(FC_ERR_INVALID, "plan is NULL");
  if (chunk_streams < 1 || depth < 1 || depth > 16)
    return fc_internal_fail(FC_ERR_INVALID, "need chunk_streams >= 1 and 1 <= depth <= 16");
  fc_pipeline* p = new fc_pipeline();
  p->plan = plan;
  p->device = fc_internal_plan_device(plan);
  p->chunk = chunk_streams;
  int rc = fc_query(plan, &p->sz);
  if (rc != FC_OK) {
    delete p;
    return rc;
  }
  DevGuard dg(p->device);
  if (!dg.ok) {
    delete p;
    return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  }
  p->ws_bytes = (size_t)chunk_streams * (size_t)p->sz.workspace_per_stream;
  cudaError_t e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
  for (int d = 0; d < depth && e == cudaSuccess; ++d) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) p->lanes.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) p->done.push_back(ev);
    // one allocation per slot: grid, wave (16-byte aligned for the float4 reductions), workspace
    const size_t g_len = (size_t)std::max(p->sz.tx_in_len, p->sz.rx_out_len);   // grid or time I/O
    const size_t sb = (size_t)p->sz.sample_bytes;
    const size_t g_b = ((size_t)chunk_streams * g_len * sb + 255) & ~(size_t)255;
    const size_t w_b = ((size_t)chunk_streams * p->sz.wave_len * sb + 255) & ~(size_t)255;
    void* m = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&m, g_b + w_b + p->ws_bytes);
    if (e == cudaSuccess) {
      p->owned.push_back(m);
      p->grid.push_back((unsigned char*)m);
      p->wave.push_back((unsigned char*)m + g_b);
      p->ws.push_back(p->ws_bytes ? (void*)((unsigned char*)m + g_b + w_b) : nullptr);
    }
  }
  if (e != cudaSuccess) {
    release(p);
    delete p;
    return cuda_err(e, "fc_pipeline_create");
  }
  *out = p;
  return FC_OK;
}

void fc_pipeline_destroy(fc_pipeline* p) {
  if (!p) return;
  {
    DevGuard dg(p->device);
    for (cudaStream_t s : p->lanes) cudaStreamSynchronize(s);
    release(p);
  }
  delete p;
}

int fc_tx_synthesize_host(fc_pipeline* pipeline, int32_t n_streams, const void* host_grid, void* host_wave,
                          void* stream) {
  FcRange nvtx_range(__func__);
  return run(pipeline, FC_TX, n_streams, host_grid, host_wave, stream);
}

int fc_rx_analyze_host(fc_pipeline* pipeline, int32_t n_streams, const void* host_wave, void* host_grid,
                       void* stream) {
  FcRange nvtx_range(__func__);
  return run(pipeline, FC_RX, n_streams, host_wave, host_grid, stream);
}

}  // extern "C"

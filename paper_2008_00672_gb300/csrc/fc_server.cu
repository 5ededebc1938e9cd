// Serving loop: slot requests of many carriers served as they arrive.
//
// Each admitted carrier owns a device-resident plan, a one-stream fc_state (so its
// slots continue one another exactly as one long frame would) and one slot of device
// input/output. A request is one slot of one carrier in one direction (TX: QAM grid ->
// waveform slot; RX: waveform slot -> QAM estimates). It is issued the moment it
// arrives — host-to-device copy, stream call, device-to-host copy, completion event —
// on its carrier's lane (a CUDA stream; carriers share lanes round-robin), so requests
// of one carrier stay in order and requests of different carriers overlap on the GPU
// with no batch boundary to wait for ("continuous batching"). Latency is measured on
// the host clock from the request's arrival to the moment its completion event is seen.
#include <chrono>
#include <cstdio>
#include <thread>
#include <vector>

#include "fc_internal.cuh"
#include "fc_trace.h"

namespace {

struct Carrier {
  fc_plan* plan = nullptr;
  fc_state* state = nullptr;
  fc_sizes sz{};
  void* d_io = nullptr;            // one allocation: grid, slot, workspace
  unsigned char* d_grid = nullptr; // fc_sizes.sample_bytes per sample
  unsigned char* d_slot = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int lane = 0;
};

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

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct fc_server {
  int device = 0;
  size_t reserve = 0;
  std::vector<cudaStream_t> lanes;
  std::vector<Carrier> carriers;
};

extern "C" {

int fc_server_create(int32_t device, int32_t n_lanes, uint64_t hbm_reserve_bytes, fc_server** out) {
  if (!out) return fc_internal_fail(FC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n_lanes < 1 || n_lanes > 128) return fc_internal_fail(FC_ERR_INVALID, "n_lanes must be 1..128");
  DevGuard dg(device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  fc_server* s = new fc_server();
  s->device = device;
  s->reserve = (size_t)hbm_reserve_bytes;
  for (int l = 0; l < n_lanes; ++l) {
    cudaStream_t st = nullptr;
    const cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t x : s->lanes) cudaStreamDestroy(x);
      delete s;
      return cuda_err(e, "cudaStreamCreate");
    }
    s->lanes.push_back(st);
  }
  *out = s;
  return FC_OK;
}

int fc_server_add_carrier(fc_server* s, const fc_geometry* geometry, int32_t* carrier_id) {
  if (!s || !geometry || !carrier_id) return fc_internal_fail(FC_ERR_INVALID, "NULL argument");
  *carrier_id = -1;
  fc_sizes sz;
  int rc = fc_geometry_check(geometry, &sz);
  if (rc != FC_OK) return rc;
  if (sz.slot_len == 0) return fc_internal_fail(FC_ERR_UNSUPPORTED, "carrier geometry cannot stream slot by slot");
  // admission: everything this carrier will hold on the device must fit in free HBM
  // minus the reserve (plan tables are bounded by a generous 8 MiB estimate)
  const size_t g_len = (size_t)(sz.tx_in_len > sz.rx_out_len ? sz.tx_in_len : sz.rx_out_len);   // grid or time I/O
  const size_t sb = (size_t)sz.sample_bytes;   // caller-facing buffers: complex64 or complex BF16
  const size_t io = align256(g_len * sb) + align256((size_t)sz.slot_len * sb) + align256((size_t)sz.workspace_per_stream);
  const size_t state = ((size_t)2 * sz.wave_len + 2 + (size_t)2 * sz.stream_delay) * 8;
  const size_t need = io + state + ((size_t)8 << 20);
  DevGuard dg(s->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemGetInfo");
  if (free_b < s->reserve || free_b - s->reserve < need) {
    char msg[200];
    snprintf(msg, sizeof msg, "admission refused: carrier needs %zu bytes, %zu free above the %zu-byte reserve", need,
             free_b > s->reserve ? free_b - s->reserve : (size_t)0, s->reserve);
    return fc_internal_fail(FC_ERR_NOMEM, msg);
  }
  Carrier c;
  c.sz = sz;
  rc = fc_plan_create(&c.plan, geometry, s->device);
  if (rc != FC_OK) return rc;
  rc = fc_state_create(c.plan, 1, &c.state);
  if (rc != FC_OK) {
    fc_plan_destroy(c.plan);
    return rc;
  }
  e = cudaMalloc(&c.d_io, io);
  if (e != cudaSuccess) {
    fc_state_destroy(c.state);
    fc_plan_destroy(c.plan);
    return cuda_err(e, "cudaMalloc of carrier buffers");
  }
  unsigned char* p = (unsigned char*)c.d_io;
  c.d_grid = p;
  c.d_slot = p + align256(g_len * sb);
  c.ws_bytes = (size_t)sz.workspace_per_stream;
  c.ws = c.ws_bytes ? (void*)(p + align256(g_len * sb) + align256((size_t)sz.slot_len * sb)) : nullptr;
  c.lane = (int)(s->carriers.size() % s->lanes.size());
  *carrier_id = (int32_t)s->carriers.size();
  s->carriers.push_back(c);
  return FC_OK;
}

int fc_server_carrier_sizes(const fc_server* s, int32_t carrier, fc_sizes* out) {
  if (!s || !out || carrier < 0 || carrier >= (int)s->carriers.size())
    return fc_internal_fail(FC_ERR_INVALID, "bad server or carrier id");
  *out = s->carriers[carrier].sz;
  return FC_OK;
}

int fc_server_run(fc_server* s, const fc_serve_request* reqs, int32_t n, double* latency_s) {
  FcRange nvtx_range(__func__);
  if (!s || (n > 0 && (!reqs || !latency_s))) return fc_internal_fail(FC_ERR_INVALID, "NULL argument");
  for (int i = 0; i < n; ++i) {
    const fc_serve_request& r = reqs[i];
    if (r.carrier < 0 || r.carrier >= (int)s->carriers.size()) return fc_internal_fail(FC_ERR_INVALID, "bad carrier");
    if (r.direction != FC_TX && r.direction != FC_RX) return fc_internal_fail(FC_ERR_INVALID, "bad direction");
    if (!r.host_in || !r.host_out) return fc_internal_fail(FC_ERR_INVALID, "request without host buffers");
    if (i > 0 && r.arrival_s < reqs[i - 1].arrival_s)
      return fc_internal_fail(FC_ERR_INVALID, "requests must be sorted by arrival time");
  }
  DevGuard dg(s->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  // one completion event per request (created up front, outside the timed loop)
  std::vector<cudaEvent_t> ev(n, nullptr);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  std::vector<int> inflight;
  inflight.reserve(n);
  int rc = FC_OK;
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
  int next = 0, done = 0;
  while (e == cudaSuccess && rc == FC_OK && done < n) {
    double t = now_s();
    while (next < n && reqs[next].arrival_s <= t && e == cudaSuccess && rc == FC_OK) {
      const fc_serve_request& r = reqs[next];
      Carrier& c = s->carriers[r.carrier];
      cudaStream_t st = s->lanes[c.lane];
      const bool tx = r.direction == FC_TX;
      unsigned char* d_in = tx ? c.d_grid : c.d_slot;
      unsigned char* d_out = tx ? c.d_slot : c.d_grid;
      const size_t sb = (size_t)c.sz.sample_bytes;
      const size_t in_b = (size_t)(tx ? c.sz.tx_in_len : c.sz.slot_len) * sb;
      const size_t out_b = (size_t)(tx ? c.sz.slot_len : c.sz.rx_out_len) * sb;
      e = cudaMemcpyAsync(d_in, r.host_in, in_b, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) break;
      rc = tx ? fc_tx_synthesize_stream(c.plan, c.state, d_in, d_out, c.ws, c.ws_bytes, (void*)st)
              : fc_rx_analyze_stream(c.plan, c.state, d_in, d_out, c.ws, c.ws_bytes, (void*)st);
      if (rc != FC_OK) break;
      e = cudaMemcpyAsync(r.host_out, d_out, out_b, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaEventRecord(ev[next], st);
      inflight.push_back(next);
      ++next;
    }
    if (e != cudaSuccess || rc != FC_OK) break;
    t = now_s();
    for (size_t k = 0; k < inflight.size();) {
      const cudaError_t q = cudaEventQuery(ev[inflight[k]]);
      if (q == cudaSuccess) {
        latency_s[inflight[k]] = t - reqs[inflight[k]].arrival_s;
        inflight[k] = inflight.back();
        inflight.pop_back();
        ++done;
      } else if (q == cudaErrorNotReady) {
        ++k;
      } else {
        e = q;
        break;
      }
    }
    if (inflight.empty() && next < n) {
      // idle until shortly before the next arrival
      const double wait = reqs[next].arrival_s - now_s();
      if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
    }
  }
  for (int l = 0; l < (int)s->lanes.size(); ++l) cudaStreamSynchronize(s->lanes[l]);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (rc != FC_OK) return rc;
  return e == cudaSuccess ? FC_OK : cuda_err(e, "fc_server_run");
}

void fc_server_destroy(fc_server* s) {
  if (!s) return;
  {
    DevGuard dg(s->device);
    for (cudaStream_t st : s->lanes) cudaStreamSynchronize(st);
    for (Carrier& c : s->carriers) {
      if (c.d_io) cudaFree(c.d_io);
      fc_state_destroy(c.state);
      fc_plan_destroy(c.plan);
    }
    for (cudaStream_t st : s->lanes) cudaStreamDestroy(st);
  }
  delete s;
}

}  // extern "C"

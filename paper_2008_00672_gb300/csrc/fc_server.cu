// Serving loop with continuous batching: slot requests of many carriers, admitted as
// they arrive and as memory frees up, and run in batches whose copies overlap the
// previous batch's compute.
//
// Each admitted carrier owns a device-resident plan and a one-stream fc_state (its slots
// continue one another exactly as one long frame would). A request is one slot of one
// carrier in one direction (TX: QAM grid -> waveform slot; RX: waveform slot -> QAM
// estimates). Its device input, output and workspace come from the server's request
// arena, a device allocation made at set-up and carved up on the host (first fit); a
// request waits in arrival order until its block fits. Requests of a carrier whose
// slot calls run in the batch's persistent launch (below) take their own frame buffer
// from the arena too, so several consecutive slots of one carrier fit in one batch;
// other requests go through the carrier's state and are admitted one per carrier and
// direction per batch.
//
// A batch runs on three CUDA streams: host-to-device copies (inputs and the batch's
// work lists), compute, device-to-host copies, joined by events, with at most
// max_inflight batches between their first copy and their last. Batches execute in
// order on the compute stream, so a carrier's slots are processed in arrival order.
// Within a batch, every symbol-synchronized complex64 carrier's slot call is one item
// list of the generic kernels' persistent launch (one launch per direction and kernel
// class, the k_sync_multi queues of the batch executor) between a batched RX prologue
// (look-behind + new slot into the request's frame; a carrier's later slots in the batch
// take their look-behind from its earlier slot's input) and a batched TX epilogue
// (carried tail added: the state's for a carrier's first slot in the batch, the earlier
// slot's frame for the next), after which one more launch moves each carrier's last carry
// into its state. Other requests run their own stream calls on the server's lanes,
// concurrently with the persistent launches.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

#include "fc_internal.cuh"
#include "fc_trace.h"

namespace {

constexpr int kMaxInflight = 8;
constexpr int kMaxChunks = 64;            // largest chunk count per stream a plan offers
constexpr int kQueues = 2 * 3 * 4;        // [direction][kernel set][occupancy class]

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Carrier {
  fc_plan* plan = nullptr;
  fc_state* state = nullptr;
  fc_sizes sz{};
  FcStateView sv{};
  size_t in_b[2] = {0, 0}, out_b[2] = {0, 0};   // per direction (FC_TX, FC_RX)
  size_t ws_b = 0;
  bool batchable = false;                       // symbol-sync, complex64: the persistent launch
  int set = 0, cls = 0;                         // its queue's kernel set and occupancy class
  size_t smem[2] = {0, 0};
};

// First-fit allocator over [0, size) in 256-byte units, on the host.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  size_t alloc(size_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, rest = it->second - n;
      free_.erase(it);
      if (rest) free_[off + n] = rest;
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t n) {
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + n == nx->first) {
      n += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += n;
        return;
      }
    }
    free_[off] = n;
  }

 private:
  std::map<size_t, size_t> free_;
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

// One batch between its first copy and its last: requests, arena blocks, the staging of
// its work lists (pinned host and device) and its events.
struct Slot {
  bool busy = false;
  int batch_id = -1;
  double admitted_s = 0;
  std::vector<int> reqs;
  std::vector<char> batched;
  std::vector<size_t> block_off, block_len;
  unsigned char* h_stage = nullptr;
  unsigned char* d_stage = nullptr;
  int* d_next = nullptr;                        // one counter per queue
  cudaEvent_t ev_in = nullptr, ev_c0 = nullptr, ev_c1 = nullptr, ev_out = nullptr, ev_fork = nullptr;
};

}  // namespace

struct fc_server {
  int device = 0;
  size_t reserve = 0;
  int num_sms = 0;
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> lane_done;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_origin = nullptr;
  std::vector<Carrier> carriers;
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0;
  Arena alloc;
  int max_batch = 64, max_inflight = 2;
  size_t stage_bytes = 0;
  Slot slots[kMaxInflight];
};

namespace {

size_t stage_bytes_for(int max_batch) {
  return align256((size_t)2 * max_batch * kMaxChunks * sizeof(FcWork)) +
         align256((size_t)max_batch * sizeof(FcSlotTx)) + align256((size_t)max_batch * sizeof(FcSlotRx)) +
         align256((size_t)2 * max_batch * sizeof(FcSlotCarry));
}

void free_slots(fc_server* s) {
  for (Slot& b : s->slots) {
    if (b.h_stage) cudaFreeHost(b.h_stage);
    if (b.d_stage) cudaFree(b.d_stage);
    if (b.d_next) cudaFree(b.d_next);
    for (cudaEvent_t ev : {b.ev_in, b.ev_c0, b.ev_c1, b.ev_out, b.ev_fork})
      if (ev) cudaEventDestroy(ev);
    b = Slot();
  }
}

cudaError_t make_slots(fc_server* s) {
  s->stage_bytes = stage_bytes_for(s->max_batch);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < s->max_inflight && e == cudaSuccess; ++i) {
    Slot& b = s->slots[i];
    e = cudaMallocHost(&b.h_stage, s->stage_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_stage, s->stage_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_next, kQueues * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b.ev_c0);
    if (e == cudaSuccess) e = cudaEventCreate(&b.ev_c1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev_fork, cudaEventDisableTiming);
  }
  return e;
}

// The arena's parts of a request, 256-byte aligned: input, output, workspace, and for a
// carrier in the persistent launch its frame (one complex64 frame of wave_len samples).
size_t request_bytes(const Carrier& c, int dir) {
  return align256(c.in_b[dir]) + align256(c.out_b[dir]) + align256(c.ws_b) +
         (c.batchable ? align256((size_t)c.sv.wave_len * sizeof(float2)) : 0);
}

// Issue one batch (its requests already admitted into slot b): copies in, compute, copies out.
int issue_batch(fc_server* s, Slot& b, const fc_serve_request* reqs) {
  const int n = (int)b.reqs.size();
  // ---- work lists on the host: persistent-launch items per queue, slot items ----
  std::vector<FcWork> work[kQueues];
  size_t qsmem[kQueues] = {};
  std::vector<FcSlotTx> stx;
  std::vector<FcSlotRx> srx;
  long long tx_max = 0, rx_max = 0;
  int n_dir[2] = {0, 0};
  for (int i = 0; i < n; ++i)
    if (b.batched[i]) ++n_dir[reqs[b.reqs[i]].direction];
  int want[2];
  for (int d = 0; d < 2; ++d) {
    // enough chunks for two CTAs per SM over the batch, no more (each chunk recomputes
    // the overlap with its neighbours)
    want[d] = n_dir[d] ? (int)std::min<long long>(kMaxChunks, (2LL * s->num_sms + n_dir[d] - 1) / n_dir[d]) : 1;
  }
  // a carrier's earlier slot in this batch (index into b.reqs, per direction), for the
  // chained carries; and its last one, for the state update
  std::map<int, int> last[2];
  std::vector<FcSlotCarry> carry[2];
  for (int i = 0; i < n; ++i) {
    if (!b.batched[i]) continue;
    const fc_serve_request& r = reqs[b.reqs[i]];
    const Carrier& c = s->carriers[r.carrier];
    unsigned char* base = s->arena + b.block_off[i];
    unsigned char* d_in = base;
    unsigned char* d_out = base + align256(c.in_b[r.direction]);
    float2* frame = (float2*)(d_out + align256(c.out_b[r.direction]) + align256(c.ws_b));
    const int q = (r.direction * 3 + c.set) * 4 + c.cls;
    const long long T = c.sv.slot_len, D = c.sv.delay;
    auto prev = last[r.direction].find(r.carrier);
    size_t smem = 0;
    if (r.direction == FC_TX) {
      fc_internal_sync_work_generic(c.plan, FC_TX, 1, d_in, frame, want[0], work[q], &smem);
      const float2* prev_tail = c.sv.tail;
      if (prev != last[0].end()) {
        const int j = prev->second;
        const Carrier& pc = s->carriers[reqs[b.reqs[j]].carrier];
        prev_tail = (const float2*)(s->arena + b.block_off[j] + align256(pc.in_b[FC_TX]) + align256(pc.out_b[FC_TX]) +
                                    align256(pc.ws_b)) + T;
      }
      stx.push_back(FcSlotTx{frame, prev_tail, (float2*)d_out, T, D});
      tx_max = std::max(tx_max, T);
    } else {
      fc_internal_sync_work_generic(c.plan, FC_RX, 1, frame, d_out, want[1], work[q], &smem);
      const float2* prev_look = c.sv.look;
      if (prev != last[1].end()) prev_look = (const float2*)(s->arena + b.block_off[prev->second]) + (T - D);
      srx.push_back(FcSlotRx{(const float2*)d_in, prev_look, frame, T, D});
      rx_max = std::max(rx_max, T + D);
    }
    last[r.direction][r.carrier] = i;
    qsmem[q] = std::max(qsmem[q], smem);
  }
  long long carry_max = 1;
  for (int d = 0; d < 2; ++d)
    for (const auto& kv : last[d]) {
      const int i = kv.second;
      const Carrier& c = s->carriers[kv.first];
      const long long T = c.sv.slot_len, D = c.sv.delay;
      unsigned char* base = s->arena + b.block_off[i];
      if (D == 0) continue;
      if (d == FC_TX) {
        const float2* frame = (const float2*)(base + align256(c.in_b[FC_TX]) + align256(c.out_b[FC_TX]) + align256(c.ws_b));
        carry[0].push_back(FcSlotCarry{frame + T, c.sv.tail, D});
      } else {
        carry[1].push_back(FcSlotCarry{(const float2*)base + (T - D), c.sv.look, D});
      }
      carry_max = std::max(carry_max, D);
    }
  size_t n_work = 0;
  for (auto& w : work) n_work += w.size();
  if (n_work > (size_t)2 * s->max_batch * kMaxChunks) return fc_internal_fail(FC_ERR_INVALID, "batch work list too long");
  // ---- staging: [work items of every queue][TX slot items][RX slot items][carries] ----
  const size_t off_tx = align256((size_t)2 * s->max_batch * kMaxChunks * sizeof(FcWork));
  const size_t off_rx = off_tx + align256((size_t)s->max_batch * sizeof(FcSlotTx));
  const size_t off_cy = off_rx + align256((size_t)s->max_batch * sizeof(FcSlotRx));
  const size_t n_cy0 = carry[0].size(), n_cy1 = carry[1].size();
  size_t qoff[kQueues];
  size_t pos = 0;
  for (int q = 0; q < kQueues; ++q) {
    qoff[q] = pos;
    if (!work[q].empty()) memcpy(b.h_stage + pos * sizeof(FcWork), work[q].data(), work[q].size() * sizeof(FcWork));
    pos += work[q].size();
  }
  if (!stx.empty()) memcpy(b.h_stage + off_tx, stx.data(), stx.size() * sizeof(FcSlotTx));
  if (!srx.empty()) memcpy(b.h_stage + off_rx, srx.data(), srx.size() * sizeof(FcSlotRx));
  if (n_cy0) memcpy(b.h_stage + off_cy, carry[0].data(), n_cy0 * sizeof(FcSlotCarry));
  if (n_cy1) memcpy(b.h_stage + off_cy + n_cy0 * sizeof(FcSlotCarry), carry[1].data(), n_cy1 * sizeof(FcSlotCarry));
  // ---- copies in ----
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const fc_serve_request& r = reqs[b.reqs[i]];
    const Carrier& c = s->carriers[r.carrier];
    e = cudaMemcpyAsync(s->arena + b.block_off[i], r.host_in, c.in_b[r.direction], cudaMemcpyHostToDevice, s->s_in);
  }
  if (e == cudaSuccess && pos)
    e = cudaMemcpyAsync(b.d_stage, b.h_stage, pos * sizeof(FcWork), cudaMemcpyHostToDevice, s->s_in);
  if (e == cudaSuccess && !stx.empty())
    e = cudaMemcpyAsync(b.d_stage + off_tx, b.h_stage + off_tx, stx.size() * sizeof(FcSlotTx), cudaMemcpyHostToDevice,
                        s->s_in);
  if (e == cudaSuccess && !srx.empty())
    e = cudaMemcpyAsync(b.d_stage + off_rx, b.h_stage + off_rx, srx.size() * sizeof(FcSlotRx), cudaMemcpyHostToDevice,
                        s->s_in);
  if (e == cudaSuccess && n_cy0 + n_cy1)
    e = cudaMemcpyAsync(b.d_stage + off_cy, b.h_stage + off_cy, (n_cy0 + n_cy1) * sizeof(FcSlotCarry),
                        cudaMemcpyHostToDevice, s->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(b.ev_in, s->s_in);
  // ---- compute: fork the lanes from the compute stream, join them back ----
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_comp, b.ev_in, 0);
  if (e == cudaSuccess) e = cudaEventRecord(b.ev_c0, s->s_comp);
  if (e == cudaSuccess) e = cudaEventRecord(b.ev_fork, s->s_comp);
  const int L = (int)s->lanes.size();
  for (int l = 0; l < L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(s->lanes[l], b.ev_fork, 0);
  if (e != cudaSuccess) return cuda_err(e, "batch copies in");
  const FcGenKernels* sets[3] = {&fc_gen_kernels_512(), &fc_gen_kernels_256(), &fc_gen_kernels_128()};
  cudaStream_t lane_tx = s->lanes[0], lane_rx = s->lanes[L > 1 ? 1 : 0];
  // RX chain: prologue, look-behind carry into the states, then the RX queues
  const FcSlotCarry* d_cy = (const FcSlotCarry*)(b.d_stage + off_cy);
  if (!srx.empty())
    e = fc_launch_slot_rx_multi((const FcSlotRx*)(b.d_stage + off_rx), (int)srx.size(), rx_max, lane_rx);
  if (e == cudaSuccess && n_cy1) e = fc_launch_slot_carry_multi(d_cy + n_cy0, (int)n_cy1, carry_max, lane_rx);
  for (int q = 0; q < kQueues && e == cudaSuccess; ++q) {
    if (work[q].empty()) continue;
    const int dir = q / 12, set = (q / 4) % 3;
    cudaStream_t st = dir == FC_TX ? lane_tx : lane_rx;
    e = sets[set]->sync_multi(dir == FC_TX, (const FcWork*)(b.d_stage + qoff[q] * sizeof(FcWork)), (int)work[q].size(), 0,
                              b.d_next + q, s->num_sms, qsmem[q], st);
  }
  // TX chain: the TX queues (above, on lane_tx), the epilogue, then the tail carry
  if (e == cudaSuccess && !stx.empty())
    e = fc_launch_slot_tx_multi((const FcSlotTx*)(b.d_stage + off_tx), (int)stx.size(), tx_max, lane_tx);
  if (e == cudaSuccess && n_cy0) e = fc_launch_slot_carry_multi(d_cy, (int)n_cy0, carry_max, lane_tx);
  if (e != cudaSuccess) return cuda_err(e, "batch persistent launch");
  // requests outside the persistent launch: their own stream calls on the other lanes
  int k = 0;
  for (int i = 0; i < n; ++i) {
    if (b.batched[i]) continue;
    const fc_serve_request& r = reqs[b.reqs[i]];
    const Carrier& c = s->carriers[r.carrier];
    cudaStream_t st = s->lanes[L > 2 ? 2 + (k++ % (L - 2)) : (k++ % L)];
    unsigned char* base = s->arena + b.block_off[i];
    unsigned char* d_in = base;
    unsigned char* d_out = base + align256(c.in_b[r.direction]);
    void* ws = c.ws_b ? (void*)(d_out + align256(c.out_b[r.direction])) : nullptr;
    const int rc = r.direction == FC_TX ? fc_tx_synthesize_stream(c.plan, c.state, d_in, d_out, ws, c.ws_b, (void*)st)
                                        : fc_rx_analyze_stream(c.plan, c.state, d_in, d_out, ws, c.ws_b, (void*)st);
    if (rc != FC_OK) return rc;
  }
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    e = cudaEventRecord(s->lane_done[l], s->lanes[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_comp, s->lane_done[l], 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b.ev_c1, s->s_comp);
  // ---- copies out ----
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_out, b.ev_c1, 0);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const fc_serve_request& r = reqs[b.reqs[i]];
    const Carrier& c = s->carriers[r.carrier];
    e = cudaMemcpyAsync(r.host_out, s->arena + b.block_off[i] + align256(c.in_b[r.direction]), c.out_b[r.direction],
                        cudaMemcpyDeviceToHost, s->s_out);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b.ev_out, s->s_out);
  return e == cudaSuccess ? FC_OK : cuda_err(e, "batch issue");
}

}  // namespace

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
  cudaError_t e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  for (int l = 0; l < n_lanes && e == cudaSuccess; ++l) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) s->lanes.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) s->lane_done.push_back(ev);
  }
  for (cudaStream_t* p : {&s->s_in, &s->s_comp, &s->s_out})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_origin);
  if (e == cudaSuccess) e = make_slots(s);
  if (e == cudaSuccess) {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    const size_t above = free_b > s->reserve ? free_b - s->reserve : 0;
    s->arena_bytes = std::min<size_t>((size_t)256 << 20, above / 2) & ~(size_t)255;
    if (e == cudaSuccess && s->arena_bytes) e = cudaMalloc(&s->arena, s->arena_bytes);
    s->alloc.reset(s->arena_bytes);
  }
  if (e != cudaSuccess) {
    fc_server_destroy(s);
    return cuda_err(e, "fc_server_create");
  }
  *out = s;
  return FC_OK;
}

int fc_server_set_limits(fc_server* s, uint64_t arena_bytes, int32_t max_batch, int32_t max_inflight) {
  if (!s) return fc_internal_fail(FC_ERR_INVALID, "server is NULL");
  if (max_batch < 1 || max_batch > 4096 || max_inflight < 1 || max_inflight > kMaxInflight)
    return fc_internal_fail(FC_ERR_INVALID, "need 1 <= max_batch <= 4096 and 1 <= max_inflight <= 8");
  const size_t want = ((size_t)arena_bytes + 255) & ~(size_t)255;
  for (const Carrier& c : s->carriers)
    for (int d = 0; d < 2; ++d)
      if (request_bytes(c, d) > want)
        return fc_internal_fail(FC_ERR_INVALID, "arena smaller than one request of an admitted carrier");
  DevGuard dg(s->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  for (cudaStream_t st : {s->s_in, s->s_comp, s->s_out}) cudaStreamSynchronize(st);
  free_slots(s);
  if (s->arena) cudaFree(s->arena);
  s->arena = nullptr;
  s->arena_bytes = 0;
  s->alloc.reset(0);
  s->max_batch = max_batch;
  s->max_inflight = max_inflight;
  cudaError_t e = make_slots(s);
  if (e != cudaSuccess) return cuda_err(e, "fc_server_set_limits (batch staging)");
  size_t free_b = 0, total_b = 0;
  e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemGetInfo");
  if (free_b < s->reserve || free_b - s->reserve < want)
    return fc_internal_fail(FC_ERR_NOMEM, "request arena does not fit above the reserve");
  if (want) {
    e = cudaMalloc(&s->arena, want);
    if (e != cudaSuccess) return cuda_err(e, "cudaMalloc of the request arena");
  }
  s->arena_bytes = want;
  s->alloc.reset(want);
  return FC_OK;
}

int fc_server_add_carrier(fc_server* s, const fc_geometry* geometry, int32_t* carrier_id) {
  if (!s || !geometry || !carrier_id) return fc_internal_fail(FC_ERR_INVALID, "NULL argument");
  *carrier_id = -1;
  fc_sizes sz;
  int rc = fc_geometry_check(geometry, &sz);
  if (rc != FC_OK) return rc;
  if (sz.slot_len == 0) return fc_internal_fail(FC_ERR_UNSUPPORTED, "carrier geometry cannot stream slot by slot");
  Carrier c;
  c.sz = sz;
  const size_t sb = (size_t)sz.sample_bytes;   // caller-facing buffers: complex64 or complex BF16
  c.in_b[FC_TX] = (size_t)sz.tx_in_len * sb;
  c.out_b[FC_TX] = (size_t)sz.slot_len * sb;
  c.in_b[FC_RX] = (size_t)sz.slot_len * sb;
  c.out_b[FC_RX] = (size_t)sz.rx_out_len * sb;
  c.ws_b = (size_t)sz.workspace_per_stream;
  // the carrier's own device memory (plan tables, bounded by a generous 8 MiB, and its
  // stream state) must fit in free HBM minus the reserve
  const size_t state = ((size_t)2 * sz.wave_len + 2 + (size_t)2 * sz.stream_delay) * 8;
  const size_t need = state + ((size_t)8 << 20);
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
  rc = fc_plan_create(&c.plan, geometry, s->device);
  if (rc != FC_OK) return rc;
  rc = fc_state_create(c.plan, 1, &c.state);
  if (rc == FC_OK) rc = fc_internal_state_view(c.state, &c.sv);
  if (rc != FC_OK) {
    fc_state_destroy(c.state);
    fc_plan_destroy(c.plan);
    return rc;
  }
  // the persistent launch takes symbol-synchronized complex64 carriers
  std::vector<FcWork> probe;
  size_t smem_tx = 0, smem_rx = 0;
  c.batchable = fc_internal_sync_work_generic(c.plan, FC_TX, 1, nullptr, nullptr, 1, probe, &smem_tx) &&
                fc_internal_sync_work_generic(c.plan, FC_RX, 1, nullptr, nullptr, 1, probe, &smem_rx);
  if (c.batchable) {
    const int threads = fc_internal_gen(c.plan).threads;
    c.set = threads == 256 ? 1 : (threads == 128 ? 2 : 0);
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device);
    const size_t per_cta = std::max(smem_tx, smem_rx) + 4096;   // + static plan copy and slack
    c.cls = (int)std::min<size_t>(4, std::max<size_t>(1, (size_t)dev_smem / per_cta)) - 1;
  }
  for (int d = 0; d < 2; ++d)
    if (request_bytes(c, d) > s->arena_bytes) {
      char msg[200];
      snprintf(msg, sizeof msg, "admission refused: a request of this carrier needs %zu bytes, the arena has %zu",
               request_bytes(c, d), s->arena_bytes);
      fc_state_destroy(c.state);
      fc_plan_destroy(c.plan);
      return fc_internal_fail(FC_ERR_NOMEM, msg);
    }
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

int fc_server_serve(fc_server* s, const fc_serve_request* reqs, int32_t n, fc_serve_record* rec) {
  FcRange nvtx_range(__func__);
  if (!s || (n > 0 && !reqs)) return fc_internal_fail(FC_ERR_INVALID, "NULL argument");
  for (int i = 0; i < n; ++i) {
    const fc_serve_request& r = reqs[i];
    if (r.carrier < 0 || r.carrier >= (int)s->carriers.size()) return fc_internal_fail(FC_ERR_INVALID, "bad carrier");
    if (r.direction != FC_TX && r.direction != FC_RX) return fc_internal_fail(FC_ERR_INVALID, "bad direction");
    if (!r.host_in || !r.host_out) return fc_internal_fail(FC_ERR_INVALID, "request without host buffers");
    if (i > 0 && r.arrival_s < reqs[i - 1].arrival_s)
      return fc_internal_fail(FC_ERR_INVALID, "requests must be sorted by arrival time");
  }
  if (n == 0) return FC_OK;
  DevGuard dg(s->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  std::vector<fc_serve_record> local;
  if (!rec) {
    local.resize(n);
    rec = local.data();
  }
  cudaError_t e = cudaEventRecord(s->ev_origin, s->s_comp);
  if (e != cudaSuccess) return cuda_err(e, "fc_server_serve");
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
  std::vector<int> pending;              // arrived, not yet in a batch, arrival order
  pending.reserve(n);
  int next = 0, done = 0, n_batches = 0, inflight = 0;
  int rc = FC_OK;
  std::vector<int> order;                // slots in issue order
  std::vector<char> in_batch(2 * s->carriers.size(), 0);
  while (rc == FC_OK && done < n) {
    double t = now_s();
    while (next < n && reqs[next].arrival_s <= t) pending.push_back(next++);
    // retire finished batches (oldest first: they finish in order)
    while (!order.empty()) {
      Slot& b = s->slots[order.front()];
      const cudaError_t q = cudaEventQuery(b.ev_out);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        rc = cuda_err(q, "batch completion");
        break;
      }
      t = now_s();
      float d0 = 0.f, d1 = 0.f;
      cudaEventElapsedTime(&d0, s->ev_origin, b.ev_c0);
      cudaEventElapsedTime(&d1, s->ev_origin, b.ev_c1);
      for (size_t i = 0; i < b.reqs.size(); ++i) {
        fc_serve_record& R = rec[b.reqs[i]];
        R.latency_s = t - reqs[b.reqs[i]].arrival_s;
        R.wait_s = b.admitted_s - reqs[b.reqs[i]].arrival_s;
        R.batch = b.batch_id;
        R.batched = b.batched[i];
        R.device_start_ms = d0;
        R.device_end_ms = d1;
        s->alloc.release(b.block_off[i], b.block_len[i]);
      }
      done += (int)b.reqs.size();
      b.busy = false;
      order.erase(order.begin());
      --inflight;
    }
    if (rc != FC_OK) break;
    // form and issue the next batch
    if (inflight < s->max_inflight && !pending.empty()) {
      int si = 0;
      while (s->slots[si].busy) ++si;
      Slot& b = s->slots[si];
      b.reqs.clear();
      b.batched.clear();
      b.block_off.clear();
      b.block_len.clear();
      std::fill(in_batch.begin(), in_batch.end(), 0);
      std::vector<int> keep;
      keep.reserve(pending.size());
      bool full = false;
      for (int idx : pending) {
        const fc_serve_request& r = reqs[idx];
        const Carrier& c = s->carriers[r.carrier];
        char& used = in_batch[2 * r.carrier + r.direction];
        size_t off = SIZE_MAX;
        const size_t len = request_bytes(c, r.direction);
        if (!full && !(used && !c.batchable) && (int)b.reqs.size() < s->max_batch) {
          off = s->alloc.alloc(len);
          if (off == SIZE_MAX) full = true;   // memory frees up as batches finish; keep the order
        }
        if (off == SIZE_MAX) {
          keep.push_back(idx);
          continue;
        }
        used = 1;
        b.reqs.push_back(idx);
        b.batched.push_back(c.batchable);
        b.block_off.push_back(off);
        b.block_len.push_back(len);
      }
      if (!b.reqs.empty()) {
        pending.swap(keep);
        b.busy = true;
        b.batch_id = n_batches++;
        b.admitted_s = now_s();
        rc = issue_batch(s, b, reqs);
        order.push_back(si);
        ++inflight;
        continue;
      }
    }
    // nothing to issue: wait for a batch to finish or for the next arrival
    if (inflight == 0 && pending.empty() && next < n) {
      const double wait = reqs[next].arrival_s - now_s();
      if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
    } else if (inflight > 0) {
      std::this_thread::yield();
    }
  }
  for (cudaStream_t st : {s->s_in, s->s_comp, s->s_out}) cudaStreamSynchronize(st);
  for (int l = 0; l < (int)s->lanes.size(); ++l) cudaStreamSynchronize(s->lanes[l]);
  for (Slot& b : s->slots) b.busy = false;
  s->alloc.reset(s->arena_bytes);
  return rc;
}

int fc_server_run(fc_server* s, const fc_serve_request* reqs, int32_t n, double* latency_s) {
  if (!s || (n > 0 && (!reqs || !latency_s))) return fc_internal_fail(FC_ERR_INVALID, "NULL argument");
  std::vector<fc_serve_record> rec(n > 0 ? n : 0);
  const int rc = fc_server_serve(s, reqs, n, rec.data());
  if (rc == FC_OK)
    for (int i = 0; i < n; ++i) latency_s[i] = rec[i].latency_s;
  return rc;
}

void fc_server_destroy(fc_server* s) {
  if (!s) return;
  {
    DevGuard dg(s->device);
    for (cudaStream_t st : s->lanes) cudaStreamSynchronize(st);
    for (cudaStream_t st : {s->s_in, s->s_comp, s->s_out})
      if (st) cudaStreamSynchronize(st);
    for (Carrier& c : s->carriers) {
      fc_state_destroy(c.state);
      fc_plan_destroy(c.plan);
    }
    free_slots(s);
    if (s->arena) cudaFree(s->arena);
    for (cudaStream_t st : s->lanes) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->lane_done) cudaEventDestroy(ev);
    for (cudaStream_t st : {s->s_in, s->s_comp, s->s_out})
      if (st) cudaStreamDestroy(st);
    if (s->ev_origin) cudaEventDestroy(s->ev_origin);
  }
  delete s;
}

}  // extern "C"

// Batch executor: a fixed list of execute calls on plans of different geometries,
// spread over internal CUDA streams ("lanes") that fork from and join into the
// caller's stream, optionally captured once into a CUDA graph and replayed.
//
// Uneven carriers (one 5 MHz carrier next to a 100 MHz one) give kernels of very
// different grid sizes; one after another, the small ones leave most of the 152 SMs
// idle and every call pays its launch latency. Side by side on lanes they fill the
// GPU together, and a graph replay issues all of them with one host call.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fc_internal.cuh"
#include "fc_trace.h"

struct fc_batch {
  int device = 0;
  std::vector<fc_batch_item> items;
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> lane_done;
  cudaStream_t origin = nullptr;                  // the stream the graph is captured on / replayed on
  cudaEvent_t ev_fork = nullptr, ev_enter = nullptr, ev_exit = nullptr;
  bool use_graph = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> owned;                       // workspaces and work lists the batch allocated
  // persistent mode: the generic symbol-sync frame calls of every item as queues of
  // (plan, stream, chunk) work items, one per direction and occupancy class (CTAs per
  // SM their shared memory allows), each run by one persistent launch
  struct Queue {
    int dir = 0;
    int io = 0;                                   // FC_IO_* bits shared by its items
    const FcGenKernels* gen = nullptr;            // kernel set (CTA size) of its items
    FcWork* d_work = nullptr;
    int n = 0;
    size_t smem = 0;
  };
  std::vector<char> in_queue;                     // item runs through a queue
  std::vector<Queue> queues;
  std::vector<void*> queue_mem;                   // work lists and counters of the queues
  int* d_next = nullptr;                          // one counter per queue
  int num_sms = 0;
  int persistent = 0;
  int want_chunks = 0;                            // chunks per stream of queued items (0: each plan's rule)
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

int run_item(const fc_batch_item& it, cudaStream_t st) {
  void* s = (void*)st;
  if (it.state) {
    return it.direction == FC_TX
               ? fc_tx_synthesize_stream(it.plan, it.state, it.in, it.out, it.workspace, it.workspace_bytes, s)
               : fc_rx_analyze_stream(it.plan, it.state, it.in, it.out, it.workspace, it.workspace_bytes, s);
  }
  return it.direction == FC_TX
             ? fc_tx_synthesize(it.plan, it.n_streams, it.in, it.out, it.workspace, it.workspace_bytes, s)
             : fc_rx_analyze(it.plan, it.n_streams, it.in, it.out, it.workspace, it.workspace_bytes, s);
}

// fork from origin, item i on lane i mod n_lanes, join back into origin
int issue(fc_batch* b) {
  cudaError_t e = cudaEventRecord(b->ev_fork, b->origin);
  for (size_t l = 0; l < b->lanes.size() && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->lanes[l], b->ev_fork, 0);
  if (e != cudaSuccess) return cuda_err(e, "batch fork");
  for (size_t q = 0; q < b->queues.size() && e == cudaSuccess; ++q) {   // the queues, on the first lanes
    const fc_batch::Queue& Q = b->queues[q];
    e = Q.gen->sync_multi(Q.dir == FC_TX, Q.d_work, Q.n, Q.io, b->d_next + q, b->num_sms, Q.smem,
                          b->lanes[q % b->lanes.size()]);
  }
  if (e != cudaSuccess) return cuda_err(e, "persistent queue launch");
  for (size_t i = 0; i < b->items.size(); ++i) {
    if (!b->in_queue.empty() && b->in_queue[i]) continue;
    const int rc = run_item(b->items[i], b->lanes[i % b->lanes.size()]);
    if (rc != FC_OK) return rc;
  }
  for (size_t l = 0; l < b->lanes.size() && e == cudaSuccess; ++l) {
    e = cudaEventRecord(b->lane_done[l], b->lanes[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->lane_done[l], 0);
  }
  return e == cudaSuccess ? FC_OK : cuda_err(e, "batch join");
}

void release(fc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaEvent_t ev : b->lane_done) cudaEventDestroy(ev);
  for (cudaEvent_t ev : {b->ev_fork, b->ev_enter, b->ev_exit})
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t s : b->lanes) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (void* p : b->owned) cudaFree(p);
  for (void* p : b->queue_mem) cudaFree(p);
}

// (Re)build the persistent work queues. Generic symbol-sync frame calls go to queues by
// direction, by I/O type (complex64 or complex BF16), by kernel set (512-, 256- or
// 128-thread CTAs) and by occupancy class (1, 2, 3 or 4 CTAs per SM for their shared
// memory), items of the largest plans first (each CTA of a launch takes the next item).
// want_chunks = 0 keeps each plan's own launch shape (calls that it runs on the
// specialised kernels stay outside the queues); want_chunks > 0 queues every complex64
// symbol-sync frame call, the one-warp-per-symbol carriers included, with that many
// chunks per stream (the plan's nearest split).
cudaError_t build_queues(fc_batch* b, int want_chunks) {
  for (void* p : b->queue_mem) cudaFree(p);
  b->queue_mem.clear();
  b->queues.clear();
  b->d_next = nullptr;
  b->in_queue.assign(b->items.size(), 0);
  b->want_chunks = want_chunks;
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b->device);
  std::vector<size_t> order(b->items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::vector<long long> size(b->items.size());
  for (size_t i = 0; i < size.size(); ++i) {
    fc_sizes sz;
    fc_query(b->items[i].plan, &sz);
    size[i] = sz.wave_len;
  }
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return size[x] > size[y]; });
  std::vector<FcWork> work[2][2][3][4];   // [direction][BF16 I/O][kernel set][occupancy class]
  size_t smem_of[2][2][3][4] = {};
  const FcGenKernels* sets[3] = {&fc_gen_kernels_512(), &fc_gen_kernels_256(), &fc_gen_kernels_128()};
  for (size_t i : order) {
    const fc_batch_item& it = b->items[i];
    if (it.state || it.n_streams == 0) continue;
    std::vector<FcWork> mine;
    size_t smem = 0;
    const bool queued =
        want_chunks > 0 && fc_internal_io(it.plan) == 0
            ? fc_internal_sync_work_generic(it.plan, it.direction, it.n_streams, it.in, it.out, want_chunks, mine, &smem)
            : fc_internal_sync_work(it.plan, it.direction, it.n_streams, it.in, it.out, mine, &smem);
    if (!queued) continue;
    const size_t per_cta = smem + 4096;                         // + static plan copy and slack
    int cls = (int)std::min<size_t>(4, std::max<size_t>(1, (size_t)dev_smem / per_cta)) - 1;
    const int bf = fc_internal_io(it.plan) != 0;
    const int set = fc_internal_gen(it.plan).threads == 256 ? 1 : (fc_internal_gen(it.plan).threads == 128 ? 2 : 0);
    b->in_queue[i] = 1;
    std::vector<FcWork>& w = work[it.direction][bf][set][cls];
    w.insert(w.end(), mine.begin(), mine.end());
    smem_of[it.direction][bf][set][cls] = std::max(smem_of[it.direction][bf][set][cls], smem);
  }
  cudaError_t e = cudaSuccess;
  for (int dir = 0; dir < 2; ++dir)
    for (int bf = 0; bf < 2; ++bf)
      for (int set = 0; set < 3; ++set)
        for (int cls = 0; cls < 4; ++cls) {
          const std::vector<FcWork>& w = work[dir][bf][set][cls];
          if (w.empty() || e != cudaSuccess) continue;
          fc_batch::Queue Q;
          Q.dir = dir;
          Q.io = bf ? (FC_IO_IN_BF16 | FC_IO_OUT_BF16) : 0;
          Q.gen = sets[set];
          Q.n = (int)w.size();
          Q.smem = smem_of[dir][bf][set][cls];
          e = cudaMalloc(&Q.d_work, w.size() * sizeof(FcWork));
          if (e == cudaSuccess) {
            b->queue_mem.push_back(Q.d_work);
            e = cudaMemcpy(Q.d_work, w.data(), w.size() * sizeof(FcWork), cudaMemcpyHostToDevice);
          }
          b->queues.push_back(Q);
        }
  if (e == cudaSuccess && !b->queues.empty()) {
    e = cudaMalloc(&b->d_next, b->queues.size() * sizeof(int));
    if (e == cudaSuccess) b->queue_mem.push_back(b->d_next);
  }
  return e;
}

}  // namespace

extern "C" {

int fc_batch_create(const fc_batch_item* items, int32_t n_items, int32_t n_lanes, int32_t mode, fc_batch** out) {
  if (!out) return fc_internal_fail(FC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!items || n_items < 1) return fc_internal_fail(FC_ERR_INVALID, "need at least one item");
  if (n_lanes < 1 || n_lanes > 64) return fc_internal_fail(FC_ERR_INVALID, "n_lanes must be 1..64");
  const int dev = fc_internal_plan_device(items[0].plan);
  for (int i = 0; i < n_items; ++i) {
    const fc_batch_item& it = items[i];
    if (!it.plan) return fc_internal_fail(FC_ERR_INVALID, "item without a plan");
    if (fc_internal_plan_device(it.plan) != dev) return fc_internal_fail(FC_ERR_INVALID, "items on different devices");
    if (it.direction != FC_TX && it.direction != FC_RX) return fc_internal_fail(FC_ERR_INVALID, "bad direction");
    if (it.n_streams < 0) return fc_internal_fail(FC_ERR_INVALID, "n_streams < 0");
  }
  DevGuard dg(dev);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  fc_batch* b = new fc_batch();
  b->device = dev;
  b->items.assign(items, items + n_items);
  b->use_graph = (mode & FC_BATCH_GRAPH) != 0;
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int l = 0; l < n_lanes && e == cudaSuccess; ++l) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->lanes.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->lane_done.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_enter, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_exit, cudaEventDisableTiming);
  // workspaces the caller left to the batch (continuous-mode plans need one per item)
  for (auto& it : b->items) {
    if (e != cudaSuccess || it.workspace) continue;
    fc_sizes sz;
    const int rc = fc_query(it.plan, &sz);
    if (rc != FC_OK) {
      release(b);
      delete b;
      return rc;
    }
    const size_t need = (size_t)it.n_streams * (size_t)sz.workspace_per_stream;
    if (need == 0) continue;
    void* p = nullptr;
    e = cudaMalloc(&p, need);
    if (e == cudaSuccess) {
      b->owned.push_back(p);
      it.workspace = p;
      it.workspace_bytes = need;
    }
  }
  if (e == cudaSuccess && (mode & FC_BATCH_PERSISTENT)) {
    b->persistent = 1;
    b->num_sms = fc_internal_num_sms(b->items[0].plan);
    e = build_queues(b, 0);
  }
  if (e != cudaSuccess) {
    release(b);
    delete b;
    return cuda_err(e, "fc_batch_create");
  }
  *out = b;
  return FC_OK;
}

int fc_batch_launch(fc_batch* b, void* stream) {
  FcRange nvtx_range(__func__);
  if (!b) return fc_internal_fail(FC_ERR_INVALID, "batch is NULL");
  DevGuard dg(b->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t caller = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(b->ev_enter, caller);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_enter, 0);
  if (e != cudaSuccess) return cuda_err(e, "batch enter");
  int rc = FC_OK;
  if (!b->use_graph) {
    rc = issue(b);
  } else {
    if (!b->exec) {
      e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_err(e, "cudaStreamBeginCapture");
      rc = issue(b);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(b->origin, &g);
      if (rc == FC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (rc != FC_OK) return rc;
      if (e != cudaSuccess) {
        b->exec = nullptr;
        return cuda_err(e, "batch graph capture");
      }
    }
    e = cudaGraphLaunch(b->exec, b->origin);
    if (e != cudaSuccess) return cuda_err(e, "cudaGraphLaunch");
  }
  if (rc != FC_OK) return rc;
  e = cudaEventRecord(b->ev_exit, b->origin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, b->ev_exit, 0);
  return e == cudaSuccess ? FC_OK : cuda_err(e, "batch exit");
}

int fc_batch_autotune(fc_batch* b, int32_t reps, void* stream) {
  FcRange nvtx_range(__func__);
  if (!b) return fc_internal_fail(FC_ERR_INVALID, "batch is NULL");
  if (reps < 1) return fc_internal_fail(FC_ERR_INVALID, "reps must be >= 1");
  DevGuard dg(b->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_enter, caller);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_enter, 0);
  // one whole pass of the batch per candidate, timed on the batch's own stream
  auto time_pass = [&](float* ms) -> int {
    for (int w = 0; w < 2; ++w) {
      const int rc = issue(b);
      if (rc != FC_OK) return rc;
    }
    cudaError_t x = cudaEventRecord(t0, b->origin);
    for (int r = 0; r < reps && x == cudaSuccess; ++r) {
      const int rc = issue(b);
      if (rc != FC_OK) return rc;
    }
    if (x == cudaSuccess) x = cudaEventRecord(t1, b->origin);
    if (x == cudaSuccess) x = cudaEventSynchronize(t1);
    if (x == cudaSuccess) x = cudaEventElapsedTime(ms, t0, t1);
    return x == cudaSuccess ? FC_OK : cuda_err(x, "batch autotune timing");
  };
  int rc = e == cudaSuccess ? FC_OK : cuda_err(e, "batch autotune");
  if (rc == FC_OK && b->persistent) {
    // the queued items' chunk count, for the mix as a whole (each plan's rule, or one
    // count for every queued item: fewer chunks recompute fewer overlapping symbols,
    // more chunks balance the launch)
    float best = 1e30f;
    int best_want = 0;
    for (int want : {0, 1, 2, 4, 8, 16, 32, 64}) {
      e = build_queues(b, want);
      if (e != cudaSuccess) {
        rc = cuda_err(e, "batch autotune queues");
        break;
      }
      float ms = 0.f;
      rc = time_pass(&ms);
      if (rc != FC_OK) break;
      if (ms < best) {
        best = ms;
        best_want = want;
      }
    }
    if (rc == FC_OK) {
      cudaStreamSynchronize(b->origin);
      e = build_queues(b, best_want);
      if (e != cudaSuccess) rc = cuda_err(e, "batch autotune queues");
    }
  } else if (rc == FC_OK) {
    // lanes: one chunk count for every frame call of the batch (each item's plan keeps it
    // as its choice for the item's stream count and direction), or the plans' own
    std::vector<int> counts = {0, 1, 2, 4, 8, 16, 32, 64};
    float best = 1e30f;
    int best_c = 0;
    std::vector<std::pair<int, int>> before(b->items.size(), {0, 0});   // each item's choice on entry
    for (size_t i = 0; i < b->items.size(); ++i) {
      const fc_batch_item& it = b->items[i];
      if (!it.state && it.n_streams > 0)
        fc_plan_choice(it.plan, it.n_streams, it.direction, &before[i].first, &before[i].second);
    }
    for (int c : counts) {
      bool any = false;
      for (size_t i = 0; i < b->items.size(); ++i) {
        const fc_batch_item& it = b->items[i];
        if (it.state || it.n_streams == 0) continue;
        fc_plan* pl = const_cast<fc_plan*>(it.plan);
        if (c > 0 && fc_plan_set_choice(pl, it.n_streams, it.direction, c, before[i].second) == FC_OK) any = true;
        else fc_plan_set_choice(pl, it.n_streams, it.direction, before[i].first, before[i].second);
      }
      if (c > 0 && !any) continue;
      float ms = 0.f;
      rc = time_pass(&ms);
      if (rc != FC_OK) break;
      if (ms < best) {
        best = ms;
        best_c = c;
      }
    }
    for (size_t i = 0; rc == FC_OK && i < b->items.size(); ++i) {
      const fc_batch_item& it = b->items[i];
      if (it.state || it.n_streams == 0) continue;
      fc_plan* pl = const_cast<fc_plan*>(it.plan);
      if (best_c == 0 || fc_plan_set_choice(pl, it.n_streams, it.direction, best_c, before[i].second) != FC_OK)
        fc_plan_set_choice(pl, it.n_streams, it.direction, before[i].first, before[i].second);
    }
  }
  cudaStreamSynchronize(b->origin);
  if (b->exec) {                          // the next launch captures the tuned batch
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (rc == FC_OK) {
    e = cudaEventRecord(b->ev_exit, b->origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, b->ev_exit, 0);
    if (e != cudaSuccess) rc = cuda_err(e, "batch autotune exit");
  }
  return rc;
}

void fc_batch_destroy(fc_batch* b) {
  if (!b) return;
  {
    DevGuard dg(b->device);
    if (b->origin) cudaStreamSynchronize(b->origin);
    release(b);
  }
  delete b;
}

}  // extern "C"

// Stream calls (fc_state): consecutive slots of one geometry processed call by call
// so that the concatenated results equal one frame of the repeated geometry.
//
// A frame of one slot is Q = T + D samples long: its last D samples overlap the next
// slot (the FC filter tails of Sec. III-B and the symbol-wise OLA of eq:multi-symb).
// When the geometry repeats with period T (same slot duration in every group, c_m T / N
// an integer so that theta_n and phi_r repeat), the K-slot frame is the sum of one-slot
// frames at offsets k T (TX), and slot k of the K-slot analysis only reads samples
// [k T, k T + Q) (RX). So a TX call runs the one-slot frame and carries D samples; an RX
// call prepends the D samples it kept from the previous input.
//
// The frame, the tail and the look-behind stay complex64 whatever the plan's I/O type:
// with FC_FLAG_IO_BF16 a TX slot (frame + tail) and an RX estimate are rounded to BF16
// once, when written to the caller's buffer, and BF16 inputs widen to FP32 exactly.
#include <cstdio>
#include <cstring>

#include <cuda_bf16.h>

#include "fc_internal.cuh"
#include "fc_trace.h"

struct fc_state {
  int device = 0;
  int n_streams = 0;
  long long wave_len = 0, slot_len = 0, delay = 0;
  float2* d_mem = nullptr;
  float2* tx_frame = nullptr;   // [n_streams][wave_len]
  float2* rx_frame = nullptr;   // [n_streams][wave_len]
  float2* tail = nullptr;       // [n_streams][delay]   TX samples [T, T + D) of the previous call
  float2* look = nullptr;       // [n_streams][delay]   last D RX input samples of the previous call
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

__device__ __forceinline__ void put(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void put(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }
__device__ __forceinline__ float2 get(const float2* p) { return *p; }
__device__ __forceinline__ float2 get(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }

// out[s][t] = frame[s][t] + tail[s][t] (t < D);  tail[s][t] = frame[s][T + t] (t < D).
// Each (s, t < D) is read and rewritten by the same thread.
template <typename TO>
__global__ void k_stream_tx(const float2* __restrict__ frame, float2* __restrict__ tail, TO* __restrict__ out,
                            long long total, long long Q, long long T, long long D) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / T, t = i - s * T;
    const float2* f = frame + s * Q;
    float2 v = f[t];
    if (t < D) {
      float2* tl = tail + s * D + t;
      const float2 c = *tl;
      v.x += c.x;
      v.y += c.y;
      *tl = f[T + t];
    }
    put(out + i, v);
  }
}

// frame[s][t] = look[s][t] (t < D) or in[s][t - D];  look[s][t] = in[s][T - D + t] (t < D).
template <typename TI>
__global__ void k_stream_rx(const TI* __restrict__ in, float2* __restrict__ look, float2* __restrict__ frame,
                            long long total, long long Q, long long T, long long D) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / Q, t = i - s * Q;
    const TI* x = in + s * T;
    if (t < D) {
      float2* lk = look + s * D + t;
      frame[i] = *lk;
      *lk = get(x + T - D + t);
    } else {
      frame[i] = get(x + t - D);
    }
  }
}

// Batched slot epilogue / prologue of the serving loop: item blockIdx.y, samples over
// blockIdx.x (grid-stride); the per-sample rules of k_stream_tx / k_stream_rx with the
// carried samples read from prev_tail / prev_look and the state updated by a later
// k_slot_carry_multi launch (the items of one launch only read what they share).
__global__ void k_slot_tx_multi(const FcSlotTx* __restrict__ items, int n) {
  const FcSlotTx it = items[blockIdx.y];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < it.T; t += (long long)gridDim.x * blockDim.x) {
    float2 v = it.frame[t];
    if (t < it.D) {
      const float2 c = it.prev_tail[t];
      v.x += c.x;
      v.y += c.y;
    }
    it.out[t] = v;
  }
}

__global__ void k_slot_rx_multi(const FcSlotRx* __restrict__ items, int n) {
  const FcSlotRx it = items[blockIdx.y];
  const long long Q = it.T + it.D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Q; t += (long long)gridDim.x * blockDim.x)
    it.frame[t] = t < it.D ? it.prev_look[t] : it.in[t - it.D];
}

__global__ void k_slot_carry_multi(const FcSlotCarry* __restrict__ items, int n) {
  const FcSlotCarry it = items[blockIdx.y];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < it.D; t += (long long)gridDim.x * blockDim.x)
    it.dst[t] = it.src[t];
}

int grid_for(long long total) {
  long long b = (total + 255) / 256;
  const long long cap = 152LL * 16;   // grid-stride beyond this
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

int check_state(const fc_plan* plan, const fc_state* st, const void* in, const void* out, fc_sizes* sz) {
  if (!plan || !st) return fc_internal_fail(FC_ERR_INVALID, "plan or state is NULL");
  int rc = fc_query(plan, sz);
  if (rc != FC_OK) return rc;
  if (sz->slot_len == 0) return fc_internal_fail(FC_ERR_UNSUPPORTED, "the plan's geometry cannot stream");
  if (sz->wave_len != st->wave_len || sz->slot_len != st->slot_len || sz->stream_delay != st->delay)
    return fc_internal_fail(FC_ERR_INVALID, "state was created for a plan with other frame sizes");
  if (fc_internal_plan_device(plan) != st->device)
    return fc_internal_fail(FC_ERR_INVALID, "state and plan are on different devices");
  if (st->n_streams == 0) return FC_OK;
  if (!in || !out) return fc_internal_fail(FC_ERR_INVALID, "input or output pointer is NULL");
  if (((uintptr_t)in | (uintptr_t)out) & (uintptr_t)(sz->sample_bytes - 1))
    return fc_internal_fail(FC_ERR_INVALID, "buffers must be aligned to the sample size (8 bytes, 4 with FC_FLAG_IO_BF16)");
  return FC_OK;
}

}  // namespace

int fc_internal_state_view(const fc_state* st, FcStateView* out) {
  if (!st || !out) return fc_internal_fail(FC_ERR_INVALID, "state is NULL");
  out->tx_frame = st->tx_frame;
  out->rx_frame = st->rx_frame;
  out->tail = st->tail;
  out->look = st->look;
  out->wave_len = st->wave_len;
  out->slot_len = st->slot_len;
  out->delay = st->delay;
  out->n_streams = st->n_streams;
  return FC_OK;
}

cudaError_t fc_launch_slot_tx_multi(const FcSlotTx* items, int n, long long max_len, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long bx = (max_len + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  k_slot_tx_multi<<<dim3((unsigned)bx, (unsigned)n), 256, 0, st>>>(items, n);
  return cudaGetLastError();
}

cudaError_t fc_launch_slot_rx_multi(const FcSlotRx* items, int n, long long max_len, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long bx = (max_len + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  k_slot_rx_multi<<<dim3((unsigned)bx, (unsigned)n), 256, 0, st>>>(items, n);
  return cudaGetLastError();
}

cudaError_t fc_launch_slot_carry_multi(const FcSlotCarry* items, int n, long long max_len, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long bx = (max_len + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  k_slot_carry_multi<<<dim3((unsigned)bx, (unsigned)n), 256, 0, st>>>(items, n);
  return cudaGetLastError();
}

extern "C" {

int fc_state_create(const fc_plan* plan, int32_t n_streams, fc_state** out) {
  if (!out) return fc_internal_fail(FC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!plan) return fc_internal_fail(FC_ERR_INVALID, "plan is NULL");
  if (n_streams < 0) return fc_internal_fail(FC_ERR_INVALID, "n_streams < 0");
  fc_sizes sz;
  int rc = fc_query(plan, &sz);
  if (rc != FC_OK) return rc;
  if (sz.slot_len == 0)
    return fc_internal_fail(FC_ERR_UNSUPPORTED,
                            "geometry cannot stream: groups differ in slot duration, some c_m T / N is not an "
                            "integer, a continuous slot is not whole hops with S_L >= L_O, or D > T");
  const int dev = fc_internal_plan_device(plan);
  DevGuard dg(dev);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  fc_state* st = new fc_state();
  st->device = dev;
  st->n_streams = n_streams;
  st->wave_len = sz.wave_len;
  st->slot_len = sz.slot_len;
  st->delay = sz.stream_delay;
  const long long S = n_streams;
  // frames first, each starting 16-byte aligned (the TX kernels reduce with float4 into
  // rows of pitch wave_len), then tail and look-behind
  const long long frame_elems = (S * sz.wave_len + 1) / 2 * 2;
  const long long elems = 2 * frame_elems + 2 * S * st->delay;
  if (elems > 0) {
    cudaError_t e = cudaMalloc(&st->d_mem, (size_t)elems * sizeof(float2));
    if (e != cudaSuccess) {
      delete st;
      return cuda_err(e, "cudaMalloc of the stream state");
    }
    // zeroed before the call returns: the caller's first stream call, or an import, may
    // come on a non-blocking stream that does not wait for the legacy default stream
    e = cudaMemset(st->d_mem, 0, (size_t)elems * sizeof(float2));
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
      cudaFree(st->d_mem);
      delete st;
      return cuda_err(e, "cudaMemset of the stream state");
    }
  }
  st->tx_frame = st->d_mem;
  st->rx_frame = st->d_mem + frame_elems;
  st->tail = st->d_mem + 2 * frame_elems;
  st->look = st->tail + S * st->delay;
  *out = st;
  return FC_OK;
}

int fc_state_reset(fc_state* state, void* stream) {
  if (!state) return fc_internal_fail(FC_ERR_INVALID, "state is NULL");
  const size_t bytes = (size_t)(2 * (long long)state->n_streams * state->delay) * sizeof(float2);
  if (bytes == 0) return FC_OK;
  DevGuard dg(state->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  const cudaError_t e = cudaMemsetAsync(state->tail, 0, bytes, (cudaStream_t)stream);
  return e == cudaSuccess ? FC_OK : cuda_err(e, "cudaMemsetAsync");
}

void fc_state_destroy(fc_state* state) {
  if (!state) return;
  {
    DevGuard dg(state->device);
    if (state->d_mem) cudaFree(state->d_mem);
  }
  delete state;
}

// A checkpoint is a 48-byte header that names the state it came from, then the device
// range [tail, tail + 2 n_streams D): every stream's TX tail, then every stream's
// look-behind (one allocation, see fc_state_create). The header lets an import refuse a
// checkpoint of another shape whose data happens to have the same byte count (two
// streams of D samples against one of 2D).
namespace {
constexpr uint32_t kCkptMagic = 0x31534346u;   // "FCS1"
struct CkptHeader {
  uint32_t magic;
  int32_t n_streams;
  int64_t delay, slot_len, wave_len;
  int64_t reserved[2];
};
static_assert(sizeof(CkptHeader) == 48, "checkpoint header layout");

CkptHeader header_of(const fc_state* st) {
  CkptHeader h{};
  h.magic = kCkptMagic;
  h.n_streams = st->n_streams;
  h.delay = st->delay;
  h.slot_len = st->slot_len;
  h.wave_len = st->wave_len;
  return h;
}
}  // namespace

int fc_state_bytes(const fc_state* state, uint64_t* bytes) {
  if (!state || !bytes) return fc_internal_fail(FC_ERR_INVALID, "state or bytes is NULL");
  *bytes = sizeof(CkptHeader) + (uint64_t)(2 * (long long)state->n_streams * state->delay) * sizeof(float2);
  return FC_OK;
}

int fc_state_export(const fc_state* state, void* host, uint64_t bytes, void* stream) {
  FcRange nvtx_range(__func__);
  uint64_t need = 0;
  const int rc = fc_state_bytes(state, &need);
  if (rc != FC_OK) return rc;
  if (!host || bytes < need) return fc_internal_fail(FC_ERR_INVALID, "host buffer missing or too small");
  const CkptHeader h = header_of(state);
  memcpy(host, &h, sizeof h);
  const uint64_t data = need - sizeof(CkptHeader);
  if (data == 0) return FC_OK;
  DevGuard dg(state->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  const cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(static_cast<unsigned char*>(host) + sizeof(CkptHeader), state->tail, (size_t)data,
                                  cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  return e == cudaSuccess ? FC_OK : cuda_err(e, "state export");
}

int fc_state_import(fc_state* state, const void* host, uint64_t bytes, void* stream) {
  FcRange nvtx_range(__func__);
  uint64_t need = 0;
  const int rc = fc_state_bytes(state, &need);
  if (rc != FC_OK) return rc;
  if (!host) return fc_internal_fail(FC_ERR_INVALID, "host is NULL");
  if (bytes != need) return fc_internal_fail(FC_ERR_INVALID, "checkpoint size does not match the state");
  CkptHeader h;
  memcpy(&h, host, sizeof h);
  const CkptHeader want = header_of(state);
  if (h.magic != kCkptMagic) return fc_internal_fail(FC_ERR_INVALID, "not a stream-state checkpoint");
  if (h.n_streams != want.n_streams || h.delay != want.delay || h.slot_len != want.slot_len ||
      h.wave_len != want.wave_len)
    return fc_internal_fail(FC_ERR_INVALID,
                            "checkpoint of another state (stream count, delay, slot or frame length differ)");
  const uint64_t data = need - sizeof(CkptHeader);
  if (data == 0) return FC_OK;
  DevGuard dg(state->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  const cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(state->tail, static_cast<const unsigned char*>(host) + sizeof(CkptHeader),
                                  (size_t)data, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  return e == cudaSuccess ? FC_OK : cuda_err(e, "state import");
}

int fc_tx_synthesize_stream(const fc_plan* plan, fc_state* state, const void* grid_in, void* slot_out,
                            void* workspace, size_t workspace_bytes, void* stream) {
  FcRange nvtx_range(__func__);
  fc_sizes sz;
  int rc = check_state(plan, state, grid_in, slot_out, &sz);
  if (rc != FC_OK || state->n_streams == 0) return rc;
  const int io = fc_internal_io(plan);
  rc = fc_internal_frame(plan, FC_TX, state->n_streams, grid_in, state->tx_frame, workspace, workspace_bytes, stream,
                         io & FC_IO_IN_BF16);
  if (rc != FC_OK) return rc;
  DevGuard dg(state->device);
  if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
  const long long total = (long long)state->n_streams * state->slot_len;
  const long long Q = sz.wave_len;
  const cudaStream_t cs = (cudaStream_t)stream;
  if (io & FC_IO_OUT_BF16)
    k_stream_tx<<<grid_for(total), 256, 0, cs>>>(state->tx_frame, state->tail, (__nv_bfloat162*)slot_out, total, Q,
                                                 state->slot_len, state->delay);
  else
    k_stream_tx<<<grid_for(total), 256, 0, cs>>>(state->tx_frame, state->tail, (float2*)slot_out, total, Q,
                                                 state->slot_len, state->delay);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FC_OK : cuda_err(e, "stream TX epilogue launch");
}

int fc_rx_analyze_stream(const fc_plan* plan, fc_state* state, const void* slot_in, void* grid_out,
                         void* workspace, size_t workspace_bytes, void* stream) {
  FcRange nvtx_range(__func__);
  fc_sizes sz;
  int rc = check_state(plan, state, slot_in, grid_out, &sz);
  if (rc != FC_OK || state->n_streams == 0) return rc;
  {
    DevGuard dg(state->device);
    if (!dg.ok) return fc_internal_fail(FC_ERR_CUDA, "cudaSetDevice failed");
    const long long Q = sz.wave_len;
    const long long total = (long long)state->n_streams * Q;
    const cudaStream_t cs = (cudaStream_t)stream;
    if (fc_internal_io(plan) & FC_IO_IN_BF16)
      k_stream_rx<<<grid_for(total), 256, 0, cs>>>((const __nv_bfloat162*)slot_in, state->look, state->rx_frame, total,
                                                   Q, state->slot_len, state->delay);
    else
      k_stream_rx<<<grid_for(total), 256, 0, cs>>>((const float2*)slot_in, state->look, state->rx_frame, total, Q,
                                                   state->slot_len, state->delay);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "stream RX prologue launch");
  }
  return fc_internal_frame(plan, FC_RX, state->n_streams, state->rx_frame, grid_out, workspace, workspace_bytes, stream,
                           fc_internal_io(plan) & FC_IO_OUT_BF16);
}

}  // extern "C"

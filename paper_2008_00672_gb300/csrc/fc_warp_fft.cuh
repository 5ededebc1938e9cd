// One-warp transforms shared by the warp-specialised kernels (fc_warp.cu,
// fc_warp_cont.cu): a warp holds 32 complex values per lane in registers and runs
// four-step FFTs of 1024 points (32 x 32) or two of 512 points (16 x 32), with one
// transpose through a padded per-warp shared-memory buffer.
#pragma once

#include <cuda_bf16.h>

#include "fc_device.cuh"
#include "fc_internal.cuh"

namespace fcwarp {
using namespace fcdev;

constexpr int kPad = 33;                       // transpose row stride in float2
constexpr int kTrans = 32 * kPad;              // per-warp transpose buffer (float2)

// Caller sample I/O: complex64, or complex BF16 ({bf16 re, bf16 im}, FC_FLAG_IO_BF16).
// The kernels compute in FP32; a BF16 output sample is rounded once, to nearest, ties
// to even, when it is stored.
using bf2 = __nv_bfloat162;
__device__ __forceinline__ float2 ld_io(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_io(const bf2* p) { return __bfloat1622float2(__ldg(p)); }
__device__ __forceinline__ void st_io(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st_io(bf2* p, float2 v) { *p = __float22bfloat162_rn(v); }

__device__ __forceinline__ void load_plan_w(FcPlanDev& P, const FcPlanDev* __restrict__ gP) {
  const int words = (int)(sizeof(FcPlanDev) / 4);
  const int* src = reinterpret_cast<const int*>(gP);
  int* dst = reinterpret_cast<int*>(&P);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
}

// exp(+j 2 pi e / n) from the forward twiddle table of size n (power of two)
__device__ __forceinline__ float2 root_pos(const float2* __restrict__ tw, int n, long long e) {
  const float2 w = __ldg(tw + (int)(e & (long long)(n - 1)));
  return make_float2(w.x, -w.y);
}

// Programmatic dependent launch: a kernel lets the next launch of its stream start its
// CTAs once all of its own CTAs are running (they are sized to be resident together);
// the next one waits for this grid's completion and memory before it touches what this
// grid writes. Without a dependent launch both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A launch, as a programmatic dependent of the stream's previous kernel when pdl is set
// (the kernels trigger their dependents at their start and wait for their
// prerequisites where they need them).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), unsigned ctas, unsigned threads, size_t smem, cudaStream_t st,
                            bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Compiler-only fence: keeps the scheduler from hoisting every load of a stage
// ahead of its first use (which would need twice the registers of the data).
__device__ __forceinline__ void sched_fence() { asm volatile("" ::: "memory"); }

// v[k] *= W^{lane e(k)} for k = 1..31 with e(k) = 4 (m & mmask) + j, k = 4 m + j.
// One 1024-point transform: tw = W_1024 table, mmask = 7 (e = k). Two 512-point
// transforms: tw = W_512 table, mmask = 3 (e = k mod 16, the same twiddles for both).
// W^{lane e} = W^{4 (m & mmask) lane} W^{j lane}: 11 table loads and one complex
// multiply per twiddle (one rounding away from the FP64-generated table; the
// table's entry 0 is exactly 1).
// STAGED: tw is instead a per-lane table in shared memory whose row e (32 float2) holds
// W^(e lane) for lane = 0..31 (rows 0..31 for 1024 points, 0..15 for 512), so that each
// twiddle is one conflict-free shared-memory read and no multiply composes it (strided
// reads tw[lane 4 m] of a plain table would hit one bank from every lane).
template <bool STAGED = false>
__device__ __forceinline__ void step_twiddles(float2 (&v)[32], const float2* __restrict__ tw, int lane, int mmask) {
  if constexpr (STAGED) {
#pragma unroll
    for (int k = 1; k < 32; ++k) v[k] = cmul(v[k], tw[((k & (4 * mmask + 3))) * 32 + lane]);
  } else {
    float2 tj[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tj[j] = __ldg(tw + lane * j);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      sched_fence();
      const float2 tm = __ldg(tw + lane * 4 * (m & mmask));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * m + j;
        if (k == 0) continue;
        v[k] = cmul(v[k], j ? cmul(tm, tj[j]) : tm);
      }
    }
  }
}

// Fill a per-lane step table for step_twiddles<true>: row e, lane l = W_n^(e l) from the
// forward table of size n (all threads of the CTA; the caller synchronises).
__device__ __forceinline__ void stage_lane_twiddles(float2* dst, const float2* __restrict__ tw, int n, int rows) {
  for (int i = threadIdx.x; i < rows * 32; i += blockDim.x) dst[i] = __ldg(tw + ((i >> 5) * (i & 31)) % n);
}

// Forward four-step FFT of one warp.
//  two512 = false: one 1024-point transform; in: lane b holds x[32 a + b] in v[a];
//                  out: lane k1 holds X[k1 + 32 k2] in v[k2].
//  two512 = true:  two 512-point transforms; in: lane b holds x_T[32 a + b] in
//                  v[16 T + a] (a < 16); out: lane k1 + 16 T holds X_T[k1 + 16 k2] in v[k2].
// STAGED: tw1024 / tw512 are per-lane step tables in shared memory (step_twiddles).
template <bool STAGED = false>
__device__ __forceinline__ void warp_fft(float2 (&v)[32], float2* scr, const float2* __restrict__ tw1024,
                                         const float2* __restrict__ tw512, int lane, bool two512) {
  if (!two512) {
    Dft<32, false>::run(v);
  } else {
    Dft<16, false>::run(v);
    Dft<16, false>::run(v + 16);
  }
  step_twiddles<STAGED>(v, two512 ? tw512 : tw1024, lane, two512 ? 3 : 7);
#pragma unroll
  for (int k = 0; k < 32; ++k) scr[k * kPad + lane] = v[k];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < 32; ++b) v[b] = scr[lane * kPad + b];
  __syncwarp();
  Dft<32, false>::run(v);
}

__device__ __forceinline__ void conj32(float2 (&v)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k].y = -v[k].y;
}

}  // namespace fcwarp

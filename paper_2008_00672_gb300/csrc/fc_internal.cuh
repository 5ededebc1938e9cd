// Internal plan layout shared by the host planner (fc_plan.cu) and the kernels
// (fc_kernels.cu). Everything a kernel needs arrives in one FcPlanDev passed by
// value; per-symbol and per-bin tables live in one device allocation.
#pragma once

#include <vector>

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fcofdm.h"

// The generic kernels (fc_kernels.cu) are compiled three times: for 512-thread CTAs, one
// per SM (transforms up to 4096 points), 256-thread CTAs, two per SM (up to 2048 points;
// fc_kernels_256.cu), and 128-thread CTAs, four per SM (up to 1024 points;
// fc_kernels_128.cu). FC_THREADS is the CTA size of the compilation at hand.
#ifndef FC_THREADS
#define FC_THREADS 512
#endif
#ifndef FC_GEN_MIN_BLOCKS
#define FC_GEN_MIN_BLOCKS 1      // resident CTAs per SM that compilation is built for
#endif
#define FC_WARP_THREADS 128      // warp-specialised kernels: 4 warps, one symbol job per warp
#ifndef FC_WARP_TX_MIN_BLOCKS
#define FC_WARP_TX_MIN_BLOCKS 2  // resident CTAs per SM the warp TX kernel is compiled for
#endif
#ifndef FC_WARP_CONT_MIN_BLOCKS
#define FC_WARP_CONT_MIN_BLOCKS 4  // resident CTAs per SM the continuous warp kernels are compiled for
#endif
#define FC_MAX_SIZES 12       // distinct transform sizes in one plan
#define FC_MAX_PASSES 8
#define FC_MAX_ELEMS_PER_THREAD 16   // in-place FFT: batch*n <= threads*16

// Elements a transform buffer of logical length n takes in shared memory: the generic
// kernels store logical element l at l + l/16 (one float2 of padding after every 16).
__host__ __device__ constexpr int fc_padded_len(int n) { return n + (n + 15) / 16; }

struct FcSize {
  int n;
  int npass;
  unsigned char radix[FC_MAX_PASSES];   // radices in pass order
  const float2* tw;   // tw[m] = exp(-j 2 pi m / n), m in [0, n), FP64-rounded
};

struct FcGroupDev {
  int N, N_O, N_S, N_L, N_T;
  int B;              // symbols
  int offset;         // placement of the group's output in the frame
  int len;            // group output length (Q or (R-1) N_S + N)
  int R;              // continuous: block count
  int size_N;         // index into FcPlanDev::sz
  int first_sub, n_sub;
  const int* sigma;   // [B] sync: sigma_n in group time
  const int* ncp;     // [B] N_CP,n
  const int* cps;     // [B] (sum_{q=1}^{n} N_CP,q) mod N
};

struct FcSubDev {
  int L, Lofdm, Lact, c, group;   // c: centre bin c_m reduced to [0, N)
  int L_S, L_L, L_T;
  int S_L;            // continuous lead pad (low rate)
  int n_low;          // continuous: low-rate stream length
  int p_lo, p_hi;     // nonzero range of D_m (shifted order)
  int size_L, size_O; // indices into sz for L and L_OFDM
  long long grid_off; // complex offset of the subband inside one stream's grid
  long long ws_off;   // complex offset inside one stream's workspace
  const float* dtx;   // [L] D_m * sqrt(I)/(sqrt(L_OFDM) N)
  const float* drx;   // [L] D_m / (sqrt(I) L sqrt(L_OFDM))
  const int* lcp;     // [B] L_CP,m,n
  const int* soff;    // [B] symbol start in the low-rate stream (CP first)
  int time_tx_off, time_rx_off;   // FC_FLAG_IO_TIME: subband offset in a stream's time I/O
};

struct FcJob {
  int group;
  int index;          // sync: symbol n; continuous: first block r0
  int nblk;           // blocks in the job (1 or 2)
  int start;          // frame time of the job's first output sample (TX) / input sample (RX)
};

struct FcChunk {
  int j0, j1;         // job range
  int t0, t1;         // TX: owned output range [t0, t1)
};

struct FcPlanDev {
  int mode, scheme_tx, scheme_rx;
  int flags;          // fc_geometry.flags
  int n_groups, n_subs, n_sizes;
  int frame_len;
  long long grid_len;
  long long ws_len;   // workspace complex elements per stream
  long long tc_off;   // tensor-core path: workspace offset of the R x 4096 spectrum rows
  int time_tx_len, time_rx_len;   // FC_FLAG_IO_TIME: per-stream time I/O lengths
  int ring;           // TX ring length (>= the longest job span and the CTA's threads)
  int ybuf;           // spectrum buffer length (complex, padded)
  int wbuf;           // low-rate buffer length (complex, padded)
  int max_span;       // longest job output span
  FcGroupDev g[FC_MAX_GROUPS];
  FcSubDev s[FC_MAX_SUBBANDS];
  FcSize sz[FC_MAX_SIZES];
};

// I/O sample type of a generic-kernel launch: complex64 unless the bit is set, then
// complex BF16 ({bf16 re, bf16 im}). A frame call of an FC_FLAG_IO_BF16 plan sets both;
// stream calls keep their internal frame in FP32 (TX: BF16 in, FP32 out; RX: the reverse).
#define FC_IO_IN_BF16 1
#define FC_IO_OUT_BF16 2

// one work item of the persistent multi-plan symbol-sync launch: one chunk of one stream
struct FcWork {
  const FcPlanDev* plan;
  const FcJob* jobs;
  const FcChunk* chunk;
  const void* in;
  void* out;
  int stream;
  int io;             // FC_IO_* bits: 0 or FC_IO_IN_BF16 | FC_IO_OUT_BF16
};
// The launchers of one compilation of the generic kernels (CTAs of `threads` threads);
// dP is the plan's device copy.
// In sync_multi every item of one launch has the same io (0 or FC_IO_IN_BF16 |
// FC_IO_OUT_BF16); set_smem_limits raises the dynamic shared-memory limit of every
// kernel of the set on the current device.
struct FcGenKernels {
  int threads;
  cudaError_t (*sync_multi)(bool tx, const FcWork* work, int n_work, int io, int* next, int num_sms, size_t smem,
                            cudaStream_t st);
  cudaError_t (*tx_sync)(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks, int n_streams,
                         const void* grid, void* wave, int io, size_t smem, cudaStream_t st);
  cudaError_t (*rx_sync)(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks, int n_streams,
                         const void* wave, void* grid, int io, size_t smem, cudaStream_t st);
  cudaError_t (*ofdm_mod)(const FcPlanDev* dP, int syms_per_stream, int n_streams, const void* grid, float2* ws,
                          int io, size_t smem, cudaStream_t st);
  cudaError_t (*tx_cont)(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks, int n_streams,
                         const float2* ws, void* wave, int io, size_t smem, cudaStream_t st);
  cudaError_t (*rx_cont)(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks, int n_streams,
                         const void* wave, float2* ws, int io, size_t smem, cudaStream_t st);
  cudaError_t (*ofdm_demod)(const FcPlanDev* dP, int syms_per_stream, int n_streams, const float2* ws, void* grid,
                            int io, size_t smem, cudaStream_t st);
  cudaError_t (*set_smem_limits)(size_t max_dynamic_smem);
};
const FcGenKernels& fc_gen_kernels_512();
const FcGenKernels& fc_gen_kernels_256();
const FcGenKernels& fc_gen_kernels_128();

// tensor-core FC passes (continuous, one subband, L = N = 4096)
#define FC_TC_TX_FFT 0
#define FC_TC_TX_IFFT 1
#define FC_TC_RX_FFT 2
#define FC_TC_RX_IFFT 3
#define FC_TC_OFDM_MOD 4     // OFDM IDFT + CP insertion into the low-rate stream (L_OFDM = 4096)
#define FC_TC_OFDM_DEMOD 5   // CP removal + OFDM DFT + active bins (overlap-save RX stream)
cudaError_t fc_launch_tc(const FcPlanDev* dP, const unsigned char* dft64, int pass, int n_streams, int n_blocks,
                         const float2* in, float2* out, float2* ws, int* err, int num_sms, cudaStream_t st,
                         unsigned first_wait = 1u << 22);
cudaError_t fc_set_tc_smem_limits();
void fc_tc_dft64_image(unsigned char* out);
size_t fc_tc_dft64_image_bytes();
// one-warp-per-symbol symbol-synchronized kernels (fc_warp.cu): the job-major item list
// of all streams (jobs: one stream's jobs in cost order) dealt to the resident CTAs; TX
// zeroes the waveform first
// weight_floats: the sum over groups of the group's subband length L (the TX weights the
// kernel stages in shared memory)
// grid_bf16 / io (FC_IO_* bits): complex-BF16 caller samples; the TX kernel accumulates
// into a complex64 waveform (zeroed here), which fc_launch_to_bf16 rounds into a BF16
// output; the RX kernel takes a complex64 waveform (fc_launch_from_bf16 widens a BF16
// one) and writes complex64 or BF16 estimates.
// TX: jobs [0, n_init) (even symbols of the only N = 2048 group, or none) initialise the
// waveform in a launch of their own; otherwise the waveform is zeroed first.
cudaError_t fc_launch_tx_sync_warp(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_init, int n_big,
                                   int n_streams, int frame_len, int weight_floats, const void* grid, int grid_bf16,
                                   float2* wave, int num_sms, cudaStream_t st);
// Jobs [0, n_big) are the N = 2048 groups' (one kernel), the rest the N = 1024 groups'
// (a second kernel: TX launches it after the first, RX before)
cudaError_t fc_launch_rx_sync_warp(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_big, int n_streams,
                                   int weight_floats, int scheme_rx, int flags, const void* wave, void* grid, int io,
                                   int num_sms, cudaStream_t st);
cudaError_t fc_launch_to_bf16(const float2* src, void* dst, long long n, int num_sms, cudaStream_t st);
cudaError_t fc_launch_from_bf16(const void* src, float2* dst, long long n, int num_sms, cudaStream_t st);
cudaError_t fc_set_warp_smem_limits();
// Continuous mode, one subband with L = L_OFDM = 384, N = 512, 50 % overlap, overlap-save
// (fc_warp_cont.cu): OFDM modulation into the workspace then FC blocks (TX), FC blocks into
// the workspace then OFDM demodulation (RX), one warp per pair of symbols or blocks.
cudaError_t fc_launch_tx_cont_warp(const FcPlanDev* dP, int n_streams, int n_symbols, int n_blocks, const void* grid,
                                   float2* ws, void* wave, int io, int num_sms, cudaStream_t st);
cudaError_t fc_launch_rx_cont_warp(const FcPlanDev* dP, int n_streams, int n_symbols, int n_blocks, const void* wave,
                                   float2* ws, void* grid, int io, int num_sms, cudaStream_t st);

// helpers for entry points defined outside fc_plan.cu
int fc_internal_fail(int code, const char* msg);     // records fc_last_error() and returns code
int fc_internal_plan_device(const fc_plan* plan);    // the device a plan was created on
int fc_internal_static_resolve(int dev);             // look up the static TX workspace on a device (fc_static.cu)
// Appends the work items of one frame call (direction FC_TX / FC_RX) on the generic
// symbol-sync kernels and returns true, or returns false when the plan's call does not
// run there (continuous mode, or the specialised kernels apply); *smem gets the call's
// dynamic shared memory.
bool fc_internal_sync_work(const fc_plan* plan, int dir, int n_streams, const void* in, void* out,
                           std::vector<FcWork>& work, size_t* smem);
// The same for a serving batch: the generic kernels whatever the plan would pick for a
// frame call (complex64 symbol-sync plans only), with the smallest chunk count per
// stream of at least want_chunks (the largest the plan has if none).
bool fc_internal_sync_work_generic(const fc_plan* plan, int dir, int n_streams, const void* in, void* out,
                                   int want_chunks, std::vector<FcWork>& work, size_t* smem);
// The generic-kernel set a plan runs on.
const FcGenKernels& fc_internal_gen(const fc_plan* plan);

// Stream-state internals for the serving loop's batched slot calls (fc_stream.cu).
struct FcStateView {
  float2* tx_frame;   // [n_streams][wave_len]
  float2* rx_frame;   // [n_streams][wave_len]
  float2* tail;       // [n_streams][delay]
  float2* look;       // [n_streams][delay]
  long long wave_len, slot_len, delay;
  int n_streams;
};
int fc_internal_state_view(const fc_state* state, FcStateView* out);
// One slot of one stream, complex64, with the carried samples given by pointer, so that
// several consecutive slots of one stream can be finished by one launch: TX epilogue
// out = frame[0, T) with prev_tail added to the first D samples (prev_tail = the state's
// tail, or the previous slot's frame + T); RX prologue frame = [prev_look; in] (prev_look
// = the state's look-behind, or the previous slot's input + T - D). FcSlotCarry then
// moves the last slot's carry into the state (dst[0, D) = src[0, D)), in a later launch.
struct FcSlotTx {
  const float2* frame;
  const float2* prev_tail;
  float2* out;
  long long T, D;
};
struct FcSlotRx {
  const float2* in;
  const float2* prev_look;
  float2* frame;
  long long T, D;
};
struct FcSlotCarry {
  const float2* src;
  float2* dst;
  long long D;
};
// One launch over n items (device arrays); max_len = the longest T (TX), T + D (RX) or D.
cudaError_t fc_launch_slot_tx_multi(const FcSlotTx* items, int n, long long max_len, cudaStream_t st);
cudaError_t fc_launch_slot_rx_multi(const FcSlotRx* items, int n, long long max_len, cudaStream_t st);
cudaError_t fc_launch_slot_carry_multi(const FcSlotCarry* items, int n, long long max_len, cudaStream_t st);
// A frame call (direction FC_TX / FC_RX) with the I/O types io (FC_IO_* bits) instead of
// the plan's own; the stream calls use it to keep their frames in FP32. Same checks and
// status as fc_tx_synthesize / fc_rx_analyze.
int fc_internal_frame(const fc_plan* plan, int dir, int n_streams, const void* in, void* out, void* workspace,
                      size_t workspace_bytes, void* stream, int io);
// The FC_IO_* bits of the plan's frame calls.
int fc_internal_io(const fc_plan* plan);
int fc_internal_num_sms(const fc_plan* plan);

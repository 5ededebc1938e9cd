/*
 * fcofdm.h -- C ABI of the GB300 fast-convolution (FC) filtered CP-OFDM library.
 *
 * The library implements the TX subband synthesis and RX subband analysis of
 * Yli-Kaakinen et al., "Frequency-Domain Signal Processing for Spectrally-
 * Enhanced CP-OFDM Waveforms in 5G New Radio":
 *   - continuous FC processing with overlap-and-add (OLA) or overlap-and-save
 *     (OLS) blocks (Sec. II and III-B, eq:BDM, eq:ola_synthesis, eq:ols_synthesis);
 *   - symbol-synchronized discontinuous FC processing with dynamic first-block
 *     overlap, CP-phase compensation theta_n, CP extrapolation and symbol-wise
 *     OLA (Sec. III-C..E, eq:padding, eq:multi-symb, eq:waveformLen);
 *   - the RX counterparts (Sec. IV, eq:ola_analysis, eq:ols_analysis, eq:concat2),
 *   - CP-OFDM modulation/demodulation of every subband (eq:TX_OFDMmod, eq:TX_CPins);
 *   - the simplified overlap-save RX of eq:reduc (FC_FLAG_REDUCED_RX).
 *
 * Around the frame calls (fc_tx_synthesize / fc_rx_analyze) the ABI offers, none of
 * it from the paper: slot-by-slot streams (fc_state), host-buffer pipelines
 * (fc_pipeline), batches of carriers of different shapes replayed as one CUDA graph
 * (fc_batch), a serving loop (fc_server), launch-shape autotuning and an
 * allocation-free TX; and as fc_geometry.flags: tensor-core transforms for 4096-point
 * carriers (FC_FLAG_TENSOR_DFT), time-domain I/O of the FC part (FC_FLAG_IO_TIME) and
 * complex-BF16 I/O buffers (FC_FLAG_IO_BF16).
 *
 * Every compute step runs in CUDA kernels for sm_103a. Nothing here falls back
 * to the CPU. All functions return an FC_* status; none throws.
 *
 * Data layout (device buffers of the frame calls, caller-owned, complex64 =
 * interleaved {float re, float im}, 8-byte aligned; 16-byte alignment recommended;
 * with FC_FLAG_IO_BF16 complex BF16 = {bfloat16 re, bfloat16 im}, 4-byte aligned):
 *   grid  [n_streams][grid_len]: per stream, subband after subband (in the
 *         order given at plan creation), [B_g][L_act,m] QAM symbols with the
 *         active subcarriers in ascending signed frequency
 *         f = -floor(L_act/2) .. ceil(L_act/2)-1 (long bin c_m + f).
 *   wave  [n_streams][wave_len]: one frame of the high-rate waveform per stream.
 *         All numerology groups are aligned so that symbol 0's cyclic prefix
 *         starts at the same sample; continuous groups start their zero-padded
 *         input S_L*I samples before that point, symbol-synchronized groups start
 *         sigma_0 = 0 at N/4 - N_CP,0 before it (eq:waveformLen).
 */
#ifndef FCOFDM_H
#define FCOFDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FC_OK 0
#define FC_ERR_INVALID 1      /* geometry or argument violates a documented constraint */
#define FC_ERR_UNSUPPORTED 2  /* valid for the paper, but a size the library has no kernel for */
#define FC_ERR_NOMEM 3        /* device allocation failed (plan creation only) */
#define FC_ERR_CUDA 4         /* a CUDA runtime call or kernel launch failed */
#define FC_ERR_TIMEOUT 5      /* a bounded device-side wait gave up */

/* processing modes (Sec. II vs Sec. III) */
#define FC_CONTINUOUS 0
#define FC_SYMBOL_SYNC 1

/* block schemes */
#define FC_OLA 0
#define FC_OLS 1

/*
 * One numerology group: subbands that share the long transform W_N and the
 * symbol timing (Sec. III: "overall symbol durations of all subband signals
 * ... have equal lengths"). Different groups get their own long transform and
 * are summed in time, x = sum_m w_m (Sec. III-B).
 */
typedef struct fc_group {
  int32_t n_long;          /* N: long (high-rate) transform size                      */
  int32_t n_overlap;       /* N_O = lambda*N high-rate overlap; symbol-sync needs N/2  */
  int32_t lead_pad;        /* continuous only: S_L*I_m in high-rate samples, -1 = N_O  */
  int32_t n_symbols;       /* B: CP-OFDM symbols per frame                             */
  const int32_t* n_cp;     /* N_CP,n, n = 0..B-1, high-rate samples (host, copied)     */
} fc_group;

/* One FC subband (Sec. II, Sec. III-A). */
typedef struct fc_subband {
  int32_t l_short;         /* L_m: short transform size, I_m = N/L_m (eqn:Rk)          */
  int32_t l_ofdm;          /* L_OFDM,m: OFDM (I)DFT size; symbol-sync needs L_OFDM = L */
  int32_t n_active;        /* L_act,m: active subcarriers                              */
  int32_t centre_bin;      /* c_m: centre bin on the long grid (may be negative)       */
  int32_t group;           /* index of the subband's numerology group                  */
  const double* weights;   /* D_m: l_short real weights, fftshifted order (index p is
                              signed bin p - floor(L/2)); host, copied at creation     */
} fc_subband;

typedef struct fc_geometry {
  int32_t mode;            /* FC_CONTINUOUS or FC_SYMBOL_SYNC                          */
  int32_t scheme_tx;       /* FC_OLA or FC_OLS                                         */
  int32_t scheme_rx;       /* FC_OLA or FC_OLS                                         */
  int32_t n_groups;        /* 1..FC_MAX_GROUPS                                         */
  const fc_group* groups;
  int32_t n_subbands;      /* 1..FC_MAX_SUBBANDS                                       */
  const fc_subband* subbands;
  int32_t flags;           /* 0, or an OR of the FC_FLAG_* bits below                  */
} fc_geometry;

/* Use the generic shared-memory kernels even where a specialised kernel exists
   (both compute the same result; this exists to test one against the other). */
#define FC_FLAG_GENERIC_KERNELS 1
/* Overlap-save symbol-synchronised RX of a subband with L_m = 1024, N_m = 2048 in the
   joint form of eq:reduc (Sec. V-A): x_hat = C Omega(g_0 - Omega g_1) + Omega Omega g_1
   with C = W S_hat W^-1, instead of the two block IDFTs, the S window, eq:concat2 and
   the OFDM DFT. Same result up to rounding. It applies to the specialised one-warp-per-
   symbol kernels with complex64 output only; other RX work (OLA, other sizes,
   FC_FLAG_GENERIC_KERNELS, complex-BF16 output) ignores it. */
#define FC_FLAG_REDUCED_RX 2
/* Continuous FC with one subband and L_m = N = 4096 (the 100 MHz NR carrier): run the
   FC block transforms on the tensor cores as a four-step GEMM-DFT (4096 = 64 x 64,
   BF16 hi/lo split, three products, FP32 accumulation), with the block steps fused
   around them; TX with OLA or OLS, RX with OLS. The result agrees with the FP32 path to
   about 1e-5 (RMS, relative). Other geometries ignore the flag. */
#define FC_FLAG_TENSOR_DFT 4
/* Time-domain I/O: TX takes, instead of the QAM grid, the low-rate CP-OFDM signal of
   every subband (per stream, subband after subband in creation order; per subband every
   symbol's L_CP,m,n samples of CP then its L_OFDM,m samples of body, true scale,
   fc_sizes.time_tx_len per stream), and RX returns, instead of QAM estimates, every
   symbol's recovered body before OFDM demodulation (per subband B_g x L_OFDM,m samples,
   fc_sizes.time_rx_len per stream). This is the FC part alone (Sec. III from eq:padding /
   eq:BDM on, Sec. IV up to eq:concat2 / CP removal), for callers with their own OFDM or
   non-OFDM signals. Runs on the generic kernels (and on the tensor-core block passes,
   whose OFDM passes it replaces by copies). */
#define FC_FLAG_IO_TIME 8
/* Complex-BF16 I/O: every caller buffer of the plan's calls (grid or time-domain input,
   waveform, slots; device and host) holds complex samples as interleaved
   {bfloat16 re, bfloat16 im}, 4 bytes a sample (fc_sizes.sample_bytes), 4-byte aligned.
   The lengths in fc_sizes are unchanged. The kernels read BF16, compute in FP32 exactly
   as without the flag, and round each output sample once to the nearest BF16 (ties to
   even): the result is the complex64 result rounded to BF16, up to the FP32 path's own
   error at rounding boundaries. Stream calls keep their TX tail and RX look-behind in
   FP32, so a streamed slot is rounded once too. Runs on the generic kernels and on the
   specialised one-warp kernels; the symbol-synchronised TX of the latter adds its
   overlapping blocks into a complex64 frame in the workspace (workspace_per_stream then
   holds one frame) and rounds it into the output in a second pass (tx_kernels = 2), and
   its RX widens the BF16 waveform into that frame first (rx_kernels = 2). The
   tensor-core kernels (FC_FLAG_TENSOR_DFT) do not apply. Combines with FC_FLAG_IO_TIME. */
#define FC_FLAG_IO_BF16 16

#define FC_MAX_GROUPS 4
#define FC_MAX_SUBBANDS 16
#define FC_MAX_TRANSFORM 4096  /* largest N, L_m or L_OFDM,m the library has kernels for */

typedef struct fc_sizes {
  int64_t grid_len;        /* complex QAM symbols per stream                           */
  int64_t wave_len;        /* complex high-rate samples per stream (one frame)         */
  int64_t nominal_len;     /* high-rate samples of the nominal duration (group 0)      */
  int64_t workspace_per_stream; /* device workspace bytes per stream for TX and RX     */
  int32_t tx_kernels;      /* kernel launches per fc_tx_synthesize                     */
  int32_t rx_kernels;      /* kernel launches per fc_rx_analyze                        */
  int64_t slot_len;        /* T: samples one stream call emits (TX) or takes (RX);
                              0 if the geometry cannot stream (see fc_state_create)    */
  int64_t stream_delay;    /* D = wave_len - slot_len: TX tail / RX look-behind length */
  int64_t time_tx_len;     /* complex samples of the time-domain TX input per stream    */
  int64_t time_rx_len;     /* complex samples of the time-domain RX output per stream   */
  int64_t tx_in_len;       /* what TX reads per stream: grid_len, or time_tx_len with
                              FC_FLAG_IO_TIME                                           */
  int64_t rx_out_len;      /* what RX writes per stream: grid_len or time_rx_len        */
  int64_t sample_bytes;    /* bytes of one complex I/O sample: 8, or 4 with FC_FLAG_IO_BF16 */
} fc_sizes;

typedef struct fc_plan fc_plan;

/*
 * Build an immutable plan: validates the geometry, derives the FC parameters
 * (eqn:Rk; L_CP,n = floor(N_CP,n L/N), Sec. III-E; sigma_n and Q,
 * eq:multi-symb / eq:waveformLen; the block map), generates twiddle, weight
 * and phase tables in FP64 on the host, rounds them once to FP32 and uploads
 * them to `device`. Allocates device memory (cudaMalloc); execute calls never
 * allocate. Returns FC_ERR_INVALID for geometry the paper's equations do not
 * define (e.g. L_O not integer, symbol-sync with lambda != 0.5 or N_CP,n > N/4,
 * continuous with a fractional low-rate CP), FC_ERR_UNSUPPORTED for transform
 * sizes outside 2^a 3^b <= FC_MAX_TRANSFORM. On error *out is NULL.
 * A plan may be used from several host threads and CUDA streams at once.
 */
int fc_plan_create(fc_plan** out, const fc_geometry* geometry, int32_t device);

/*
 * Host-only validation: runs every check of fc_plan_create and fills `out`
 * (may be NULL) without touching a GPU or allocating device memory.
 */
int fc_geometry_check(const fc_geometry* geometry, fc_sizes* out);

/* Per-stream sizes of the buffers an execute call reads and writes. */
int fc_query(const fc_plan* plan, fc_sizes* out);

/*
 * TX subband synthesis (Sec. III): grid [n_streams][grid_len] -> wave
 * [n_streams][wave_len]. CP-OFDM modulation, FC blocks (short DFT, fftshift,
 * D_m, bin map with phi_r theta_n, sqrt(I_m)-scaled long IDFT), OLA/OLS and
 * symbol-wise assembly, sum over subbands and groups. Every wave sample is
 * written (no pre-zeroing needed). `workspace` (device, >= n_streams *
 * workspace_per_stream bytes, may be NULL when that is 0) holds the low-rate
 * CP-OFDM stream of continuous mode. Asynchronous on `stream` (a cudaStream_t,
 * NULL = default stream); buffers must stay valid until the stream reaches it.
 * n_streams == 0 is a no-op.
 */
int fc_tx_synthesize(const fc_plan* plan, int32_t n_streams, const void* grid_in, void* wave_out,
                     void* workspace, size_t workspace_bytes, void* stream);

/*
 * RX subband analysis (Sec. IV): wave [n_streams][wave_len] -> grid
 * [n_streams][grid_len] (QAM estimates on the active subcarriers): long DFT,
 * bin gather with conj(phi_r theta_n), D_m, inverse shift, 1/sqrt(I_m)-scaled
 * short IDFT, OLS discard or OLA accumulate, concatenation / CP removal
 * (eq:concat2) and OFDM demodulation. Same buffer rules as fc_tx_synthesize.
 */
int fc_rx_analyze(const fc_plan* plan, int32_t n_streams, const void* wave_in, void* grid_out,
                  void* workspace, size_t workspace_bytes, void* stream);

/*
 * Stream calls: a stream is an endless sequence of slots of this geometry (a slot =
 * the CP lists of all groups, duration T = fc_sizes.slot_len samples). The paper
 * processes one frame with zero history (Sec. III-B pads both ends, eq:waveformLen
 * sizes the symbol-synchronized frame); a stream call instead continues the previous
 * call, so that K calls give exactly what one frame of the K-slot geometry (every
 * CP list repeated K times, slot grids stacked per subband) gives:
 *   TX: the concatenated outputs of calls 0..K-1 are samples [0, K T) of the K-slot
 *       frame (its last D = fc_sizes.stream_delay samples stay in the state and come
 *       out at the start of call K).
 *   RX: call k decodes slot k from the D samples before its input (the "look-behind",
 *       kept in the state) followed by its T input samples, i.e. from samples
 *       [k T, k T + Q) of the stream [look-behind at reset; input 0; input 1; ...].
 *       The K-slot frame x (length K T + D) is decoded by a priming call whose input
 *       ends with x[0, D) (its output discarded) and then calls on x[D + k T, D + (k+1) T).
 * This holds exactly (up to rounding) when every group lasts the same T, every
 * c_m T / N_m is an integer (theta_n and phi_r then repeat every slot; true for the
 * 5G NR numerologies, where the CPs of a slot add up to whole symbols) and, in
 * continuous mode, T L_m / N_m is a whole number of hops L_S with S_L >= L_O; and
 * D <= T. Otherwise slot_len is 0 and fc_state_create returns FC_ERR_UNSUPPORTED.
 *
 * fc_state holds, per stream, the TX tail and the RX look-behind (D samples each,
 * zero at creation) and one frame buffer per direction. It is created for a fixed
 * n_streams and may be used with any plan of the same device whose fc_sizes give the
 * same wave_len, slot_len and stream_delay. TX calls of one state must be ordered
 * (same CUDA stream, or synchronised), and so must its RX calls; a TX and an RX call
 * of one state may overlap (they touch disjoint buffers).
 */
typedef struct fc_state fc_state;

/* Allocates the state on the plan's device (cudaMalloc; the stream calls never
   allocate). FC_ERR_UNSUPPORTED if the plan's geometry cannot stream. */
int fc_state_create(const fc_plan* plan, int32_t n_streams, fc_state** out);

/* Zeroes the TX tail and the RX look-behind, asynchronously on `stream`. */
int fc_state_reset(fc_state* state, void* stream);

/* Frees the state (after its calls have finished). Safe on NULL. */
void fc_state_destroy(fc_state* state);

/*
 * Checkpoint / resume (no counterpart in the paper). A stream's whole state is its TX
 * tail and RX look-behind: D = fc_sizes.stream_delay complex64 samples each per stream.
 * fc_state_bytes gives the size of a checkpoint: a 48-byte header (a magic word, the
 * stream count, D, the slot and frame lengths of the state that wrote it), then
 * 2 x n_streams x D x 8 bytes (every stream's TX tail, then every stream's
 * look-behind). fc_state_export waits for the work queued on `stream` (a cudaStream_t,
 * NULL = default stream) and copies the state into `host` (at least that many bytes,
 * host memory, caller-owned). fc_state_import copies a checkpoint of exactly that size
 * into a state created for a plan of the same geometry and the same number of streams,
 * in order on `stream`, complete when the call returns. A stream resumed from a
 * checkpoint continues as the one that wrote it. FC_ERR_INVALID for NULL arguments, a
 * wrong size, or a header that does not match the state (another stream count, D,
 * slot or frame length); FC_ERR_CUDA if a copy fails.
 */
int fc_state_bytes(const fc_state* state, uint64_t* bytes);
int fc_state_export(const fc_state* state, void* host, uint64_t bytes, void* stream);
int fc_state_import(fc_state* state, const void* host, uint64_t bytes, void* stream);

/*
 * One TX stream call: grid [n_streams][grid_len] -> slot_out [n_streams][slot_len].
 * Runs fc_tx_synthesize into the state's frame buffer, then adds the carried tail to
 * the first D samples and keeps samples [T, T + D) as the next tail. Workspace and
 * stream rules as fc_tx_synthesize; n_streams is the state's.
 */
int fc_tx_synthesize_stream(const fc_plan* plan, fc_state* state, const void* grid_in, void* slot_out,
                            void* workspace, size_t workspace_bytes, void* stream);

/*
 * One RX stream call: slot_in [n_streams][slot_len] -> grid [n_streams][grid_len].
 * Assembles [look-behind; slot_in] in the state's frame buffer, keeps the last D
 * input samples as the next look-behind and runs fc_rx_analyze on the frame.
 */
int fc_rx_analyze_stream(const fc_plan* plan, fc_state* state, const void* slot_in, void* grid_out,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * Allocation-free TX (no counterpart in the paper; it is a deployment option).
 * Same computation and buffer rules as fc_tx_synthesize, but the workspace is a
 * device array built into the library (FC_STATIC_WORKSPACE_BYTES per GPU) instead
 * of a caller buffer, for callers that cannot allocate device memory at run time
 * (fixed-budget real-time loops, hosts whose allocator belongs to another
 * framework). The call never calls cudaMalloc/cudaFree or any allocating routine.
 *  - The array is reserved on a GPU when the first plan is created there
 *    (fc_plan_create looks up its device address with that device current) and held
 *    until the process exits. If that reservation failed, the first call of this
 *    entry point tries again and returns FC_ERR_NOMEM when the GPU has no room.
 *    Make that first call before capturing the stream into a CUDA graph.
 *  - Returns FC_ERR_INVALID (see fc_last_error) if n_streams * workspace_per_stream
 *    exceeds FC_STATIC_WORKSPACE_BYTES; plans with no workspace need (symbol-sync
 *    mode) are not limited.
 *  - The array's address is kept per device for the life of the process, so
 *    cudaDeviceReset (or releasing the primary context) is not supported while the
 *    library is in use.
 *  - All calls on one device share the one array: calls that overlap on the GPU
 *    (different CUDA streams, or several host threads) race and corrupt each
 *    other's output. Serialise them. Nothing in the array needs clearing between
 *    calls; each call writes every element it reads.
 */
#define FC_STATIC_WORKSPACE_BYTES (32u << 20)
int fc_tx_synthesize_static(const fc_plan* plan, int32_t n_streams, const void* grid_in, void* wave_out,
                            void* stream);

/* FC_OK, or FC_ERR_TIMEOUT once if a tensor-core kernel of this plan gave up a bounded
   wait since the last call (its output is then wrong). Synchronous: reads one device
   word. */
int fc_plan_device_status(const fc_plan* plan);

/* Test hook of the bounded waits (no counterpart in the paper). Sets how many times
   each CTA of this plan's tensor-core kernels polls its first GEMM-completion mbarrier
   before it gives up (default 2^22, the limit every other wait keeps). With 0 the first
   wait gives up at once: the CTA records the failure, waits (with the default limit)
   for its copy and GEMM in flight, releases its tensor memory and returns, so the next
   fc_plan_device_status reports FC_ERR_TIMEOUT and the call's output is wrong; the plan
   stays usable. Not to be changed while a call of the plan is being issued.
   FC_ERR_INVALID for a NULL plan. */
int fc_plan_set_first_wait_limit(fc_plan* plan, uint32_t polls);

/* Directions, for the autotuner and the batch executor. */
#define FC_TX 0
#define FC_RX 1

/*
 * Autotuner (no counterpart in the paper; launch-shape selection on this GPU). For
 * n_streams streams, times every launch shape the plan has for TX and for RX: the
 * specialised kernels where the plan has them (one shape: the one-warp-per-symbol
 * kernels deal all streams' symbol jobs to the CTAs resident on the GPU; the tensor-
 * core passes one tile of two transforms per CTA step), and the generic shared-memory
 * kernels at every number of CTAs each stream's symbol jobs are spread over (1, 2,
 * 4, ... chunks per stream) and every CTA size that fits the plan (512 threads one per
 * SM, 256 two per SM, 128 four per SM). Each runs `reps` times on `stream`; the
 * fastest per direction is recorded in the plan. Later execute calls with exactly
 * n_streams streams use it; other counts keep the built-in rule (the specialised
 * kernels where the plan has them; else chunks so that the call launches at least two
 * CTAs per SM, 128-thread CTAs where the call fills four per SM, else 256-thread CTAs
 * where they fit). Then, when a chosen shape runs the generic kernels, it tunes their
 * radix schedules: for each transform size of the plan in turn, each candidate
 * schedule (fc_plan_radices) is timed on those directions and the fastest is written
 * into the plan's device tables, where every later generic launch of the plan reads it
 * (whatever its stream count). Results do not depend on the choice beyond rounding.
 * Allocates and frees temporary device buffers and synchronises `stream`: call it at
 * set-up, not inside a stream capture or while calls of the plan are in flight.
 */
int fc_plan_autotune(fc_plan* plan, int32_t n_streams, int32_t reps, void* stream);

/* The radix schedule of the plan's n-point transform on the generic kernels: passes in
   order (radices 2, 3, 4, 8, 16; their product is n) into radices[0 .. *n_passes),
   which must hold 8 entries. Built-in rule: every factor 3 as a radix-3 pass, last; the
   power of two in ceil(a/4) balanced passes of at most radix 16, larger first; the
   autotuner may change it. FC_ERR_INVALID when the plan has no n-point transform. */
int fc_plan_radices(const fc_plan* plan, int32_t n, int32_t* radices, int32_t* n_passes);

/* Records a launch shape for n_streams streams in `direction` without timing (e.g. one
   saved from an earlier fc_plan_autotune): chunks_per_stream must be one the plan has
   (1, 2, 4, ..., at most 64 and at most the jobs per stream); generic_kernels 1 selects
   the generic shared-memory kernels where specialised ones exist (their CTA size then
   follows the built-in rule), and chunks_per_stream applies to the generic kernels only
   (the specialised ones have a single shape). FC_ERR_INVALID otherwise. */
int fc_plan_set_choice(fc_plan* plan, int32_t n_streams, int32_t direction, int32_t chunks_per_stream,
                       int32_t generic_kernels);

/* The launch shape an execute call with n_streams streams will use in `direction`. */
int fc_plan_choice(const fc_plan* plan, int32_t n_streams, int32_t direction, int32_t* chunks_per_stream,
                   int32_t* generic_kernels);

/*
 * Batch executor (no counterpart in the paper). Runs a fixed list of execute calls on
 * plans of different geometries (carriers with their own bandwidth, numerology and
 * subbands) as one unit: the calls are spread over `n_lanes` internal CUDA streams
 * that fork from and join back into the caller's stream, so small carriers run side
 * by side instead of one after another. With FC_BATCH_GRAPH the first fc_batch_launch
 * captures the whole fork/join into a CUDA graph and later launches replay it (one
 * host call for every kernel of every item); the items' pointers are then fixed, so
 * refill the same buffers between launches. With FC_BATCH_PERSISTENT the items that
 * run on the generic symbol-sync kernels share one persistent launch per direction. Items with a state are stream calls
 * (fc_tx_synthesize_stream / fc_rx_analyze_stream), others frame calls. Items must
 * not share output buffers, workspaces or states. Every item's result equals that of
 * its own call.
 */
typedef struct fc_batch_item {
  const fc_plan* plan;
  fc_state* state;           /* NULL: frame call                                        */
  int32_t direction;         /* FC_TX or FC_RX                                          */
  int32_t n_streams;         /* must be the state's n_streams when state != NULL        */
  const void* in;            /* device: grid (TX) or waveform / slot (RX)               */
  void* out;                 /* device: waveform / slot (TX) or grid (RX)               */
  void* workspace;           /* device, or NULL: the batch allocates what the plan needs */
  size_t workspace_bytes;
} fc_batch_item;

typedef struct fc_batch fc_batch;

/* mode bits of fc_batch_create */
#define FC_BATCH_GRAPH 1       /* capture the first launch into a CUDA graph, replay it after */
#define FC_BATCH_PERSISTENT 2  /* frame calls that run on the generic symbol-sync kernels go into one
                                  work queue per direction (one item = one chunk of one stream),
                                  run by one persistent launch that takes items largest plan first */

/* Copies the item list; allocates the lanes, events, missing workspaces and (with
   FC_BATCH_PERSISTENT) the work queues. `mode` is an OR of the FC_BATCH_* bits. */
int fc_batch_create(const fc_batch_item* items, int32_t n_items, int32_t n_lanes, int32_t mode, fc_batch** out);
int fc_batch_launch(fc_batch* batch, void* stream);

/* Autotuner of the batch as a whole (no counterpart in the paper): times reps passes of
   the whole batch (its work, not a graph replay; on internal streams ordered after the
   caller's `stream`) for each candidate and keeps the fastest for the mix, where tuning
   each carrier alone does not find it. With FC_BATCH_PERSISTENT the candidates are the
   queued items' chunks per stream (each plan's own rule, or one count 1..64 for every
   complex64 symbol-synchronized frame call, which also puts the one-warp-per-symbol
   carriers into the queues); otherwise one chunk count for every frame call, which each
   item's plan keeps as its choice for that stream count and direction. A captured graph
   is dropped and recaptured by the next fc_batch_launch. Returns when done. */
int fc_batch_autotune(fc_batch* batch, int32_t reps, void* stream);
void fc_batch_destroy(fc_batch* batch);

/*
 * Serving loop (no counterpart in the paper; the deployment around the FC path).
 * A server holds admitted carriers, each with a device-resident plan and a one-stream
 * fc_state (the TX tail and RX look-behind that join consecutive slots), and serves
 * slot requests of those carriers as they arrive, with continuous batching:
 *  - A request is admitted when its input, output and workspace fit in the server's
 *    request arena (device memory reserved by fc_server_set_limits) and no request of
 *    the same carrier and direction is already in the batch being formed; admitted
 *    requests wait in arrival order otherwise. Its arena space is freed when its output
 *    has reached the host.
 *  - Whenever fewer than max_inflight batches are on the device, the admitted requests
 *    form the next batch (at most max_batch): their host-to-device copies on one CUDA
 *    stream, their compute on a second, their device-to-host copies on a third, so
 *    a batch's copies overlap the previous batch's compute. Within a batch, the slot
 *    calls of every symbol-synchronized complex64 carrier run together: one persistent
 *    launch of the generic kernels per direction and kernel class over all of them, with
 *    one batched TX epilogue and one batched RX prologue around it. Other requests
 *    (continuous mode, tensor-core and complex-BF16 carriers) run their own stream calls
 *    on the server's lanes inside the same batch, concurrently with it.
 *  - Requests of one carrier and direction run in arrival order (batches execute in
 *    order on the compute stream), so each carrier's results equal its own stream calls
 *    whatever else the server is doing.
 * Latency is measured on the host clock from a request's arrival to the moment its
 * batch's completion event is seen.
 */
typedef struct fc_server fc_server;

typedef struct fc_serve_request {
  double arrival_s;        /* seconds after the start of fc_server_run; non-decreasing  */
  int32_t carrier;         /* id from fc_server_add_carrier                             */
  int32_t direction;       /* FC_TX: grid in, slot_len samples out; FC_RX: the reverse  */
  const void* host_in;     /* host samples, complex64 or (FC_FLAG_IO_BF16) complex BF16;
                              page-locked memory for asynchronous copies                */
  void* host_out;
} fc_serve_request;

/* What fc_server_serve reports per request. */
typedef struct fc_serve_record {
  double latency_s;        /* arrival to observed completion (host clock)                */
  double wait_s;           /* arrival to admission into a batch (host clock)             */
  int32_t batch;           /* index of the batch it ran in                               */
  int32_t batched;         /* 1: in the batch's persistent launch; 0: its own stream call */
  float device_start_ms;   /* the batch's compute interval on the device (CUDA events),  */
  float device_end_ms;     /*   relative to the start of the first batch's compute       */
} fc_serve_record;

/* n_lanes CUDA streams; admission keeps hbm_reserve_bytes of device memory free. The
   request arena starts at min(256 MiB, free memory above the reserve / 2); max_batch 64,
   max_inflight 2. */
int fc_server_create(int32_t device, int32_t n_lanes, uint64_t hbm_reserve_bytes, fc_server** out);

/* Sets the request arena (device bytes for the inputs, outputs and workspaces of
   admitted requests; reallocated here, never during serving), the largest batch and the
   number of batches on the device at once (1..8). FC_ERR_NOMEM when the arena does not
   fit above the reserve; FC_ERR_INVALID for out-of-range values. Not while serving. */
int fc_server_set_limits(fc_server* server, uint64_t arena_bytes, int32_t max_batch, int32_t max_inflight);

/* Admits a carrier (its geometry must stream: fc_sizes.slot_len > 0). FC_ERR_NOMEM,
   with nothing allocated, when its plan and state would not fit in the free device
   memory above the reserve, or when one of its requests could never fit in the arena. */
int fc_server_add_carrier(fc_server* server, const fc_geometry* geometry, int32_t* carrier_id);

/* The sizes of an admitted carrier (grid_len, slot_len, ...). */
int fc_server_carrier_sizes(const fc_server* server, int32_t carrier, fc_sizes* out);

/* Replays `requests` (sorted by arrival) in real time; records[i] (may be NULL) gets
   request i's latency, wait, batch and device interval. Returns when every request has
   completed. Host output buffers of one carrier and direction may be shared between
   requests only if the caller does not need the earlier results. */
int fc_server_serve(fc_server* server, const fc_serve_request* requests, int32_t n_requests,
                    fc_serve_record* records);

/* fc_server_serve reporting only the latencies (seconds) into latency_s. */
int fc_server_run(fc_server* server, const fc_serve_request* requests, int32_t n_requests, double* latency_s);

/* Frees every carrier and the lanes (after synchronising them). Safe on NULL. */
void fc_server_destroy(fc_server* server);

/*
 * Host-buffer execute calls (no counterpart in the paper; how a host application feeds
 * the path). A pipeline owns `depth` slots of device buffers for `chunk_streams` streams
 * (input, output, workspace) and one CUDA stream per slot; fc_tx_synthesize_host /
 * fc_rx_analyze_host split n_streams into chunks, and chunk i copies its host input to
 * slot i mod depth, runs fc_tx_synthesize / fc_rx_analyze there and copies the result
 * back, on that slot's CUDA stream. Copies in both directions and the kernels of
 * different chunks therefore overlap. The calls are asynchronous with respect to the
 * host (ordered after earlier work on `stream`, and later work on `stream` waits for
 * them); host buffers must stay valid until then and should be page-locked (pageable
 * memory makes the copies synchronous and removes the overlap). Results equal the
 * device calls on the same data. A pipeline serves one call at a time: order calls on
 * the same pipeline through one `stream`.
 */
typedef struct fc_pipeline fc_pipeline;

/* Allocates depth x (grid + wave + workspace for chunk_streams streams) on the plan's
   device; 1 <= depth <= 16. The plan must outlive the pipeline. */
int fc_pipeline_create(const fc_plan* plan, int32_t chunk_streams, int32_t depth, fc_pipeline** out);
void fc_pipeline_destroy(fc_pipeline* pipeline);

/* host grid [n_streams][grid_len] -> host wave [n_streams][wave_len] */
int fc_tx_synthesize_host(fc_pipeline* pipeline, int32_t n_streams, const void* host_grid, void* host_wave,
                          void* stream);
/* host wave [n_streams][wave_len] -> host grid [n_streams][grid_len] */
int fc_rx_analyze_host(fc_pipeline* pipeline, int32_t n_streams, const void* host_wave, void* host_grid,
                       void* stream);

/* Frees the plan's device tables. Safe on NULL. Must not race with running calls. */
void fc_plan_destroy(fc_plan* plan);

/* Human-readable text for a status code (static storage). */
const char* fc_status_string(int status);

/* Text of the last error recorded on this host thread (static per thread). */
const char* fc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FCOFDM_H */

// FC blocks on the 5th-generation tensor cores (tcgen05): the 4096-point short and
// long DFTs of continuous FC with L = N = 4096 (Sec. III-B, eq:BDM; the 100 MHz NR
// carrier) as a four-step GEMM-DFT, 4096 = 64 x 64.
//
//   X[k1 + 64 k2] = sum_n2 W64^(n2 k2) W4096^(n2 k1) sum_n1 W64^(n1 k1) x[64 n1 + n2]
//
// Stage 1 multiplies the 64 x 64 data matrix by the DFT-64 matrix, the twiddles
// W4096^(n2 k1) are applied in registers, stage 3 multiplies by the DFT-64 matrix
// again. Complex numbers ride along K and N as interleaved (re, im) pairs: the data
// rows are the M side (A, K-major, (re, im) of 64 inputs = K 128), the DFT-64 matrix
// is the B side (N 128 = (re, im) of 64 outputs), so D = A B^T gives each TMEM lane
// (one data row) its 64 complex outputs side by side.
//
// Precision: BF16 operands split as x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and
// three products hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM: about 16 bits of
// each operand reach the product (relative error ~1e-5 per transform), far below the
// -60 dB budget of the reduced-precision path.
//
// One CTA (512 threads, 16 warps) per SM works through tiles of two transforms
// (M = 128 rows): every thread stages operands into shared memory (128-byte swizzle,
// the layout the MMA descriptors name), one thread issues the MMAs, warps read the
// accumulator back with tcgen05.ld. The FC steps around the transforms are fused into
// the operand staging (prologue: segmentation, A window, conjugation) and the
// accumulator read-back (epilogue: shift, D_m, phi_r, bin map, OLA / OLS assembly).
// The transform between two passes goes through the workspace.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>

#include "fc_device.cuh"
#include "fc_internal.cuh"
#include "fc_tc.cuh"

namespace {

using namespace fcdev;
using namespace fctc;

constexpr int kN = 4096;
constexpr int kThreads = 512;
constexpr int kChunk = 128 * 128;          // bytes of one 64-element K chunk of a 128-row operand
constexpr int kOp = 2 * kChunk;            // one 128 x 128 BF16 operand (K = 128): 32 KB
constexpr int kStage = 2 * 4096 * 8;      // FP32 input of the next tile (two transforms): 64 KB
constexpr int kSmem = 4 * kOp + kStage + 1024;   // B hi, B lo, A hi, A lo, staging, alignment slack
constexpr uint32_t kIdesc =                // kind::f16, BF16 x BF16 -> FP32, K-major, M = N = 128
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

// Byte offset of BF16 element k of row `row` in a 128-row, K = 128 operand: two
// 64-element chunks, rows of 128 bytes, 16-byte units XOR-swizzled by row % 8.
__host__ __device__ __forceinline__ uint32_t op_off(int row, int k) {
  const int j = k >> 6, byte = (k & 63) * 2;
  return (uint32_t)(j * kChunk + row * 128 + ((((byte >> 4) ^ (row & 7))) << 4) + (byte & 15));
}

// v = hi + lo in BF16 pairs, returned as the 32-bit words the operand stores
__device__ __forceinline__ void split_pack(float2 v, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, uint32_t off, float2 v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat162*>(lo + off) = l;
}

// exp(+j 2 pi e / n) from the table W_n^m = exp(-j 2 pi m / n), n a power of two
__device__ __forceinline__ float2 root_pos_tc(const float2* __restrict__ tw, int n, long long e) {
  const float2 w = __ldg(tw + (int)(e & (long long)(n - 1)));
  return make_float2(w.x, -w.y);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct TcArgs {
  const FcPlanDev* P;
  const unsigned char* dft64;   // B operand images: hi then lo (kOp bytes each)
  int pass;                     // FC_TC_TX_FFT, FC_TC_TX_IFFT, FC_TC_RX_FFT, FC_TC_RX_IFFT
  int n_streams;
  const float2* in;             // wave (RX_FFT) or workspace
  float2* out;                  // wave (TX_IFFT) or workspace
  float2* ws;                   // workspace base
  int* err;                     // set to 1 when a bounded wait gives up
  unsigned first_wait;          // poll limit of each CTA's first GEMM-completion wait
};

// FC parameters of the one subband, read once per CTA into registers (reading them
// through the plan pointer would reload them after every store the compiler cannot
// prove disjoint).
struct TcK {
  long long ws_len, ws_off, tc_off, frame_len, offset, grid_len, grid_off;
  int N_S, N_L, R, L_L, L_S, S_L, n_low, c, Lact, B;
  bool ola_tx;
  const float* __restrict__ dtx;
  const float* __restrict__ drx;
  const int* __restrict__ lcp;
  const int* __restrict__ soff;
};

__device__ __forceinline__ TcK tc_consts(const FcPlanDev& P) {
  const FcGroupDev& G = P.g[0];
  const FcSubDev& S = P.s[0];
  TcK k;
  k.ws_len = P.ws_len; k.ws_off = S.ws_off; k.tc_off = P.tc_off; k.frame_len = P.frame_len; k.offset = G.offset;
  k.grid_len = P.grid_len; k.grid_off = S.grid_off;
  k.N_S = G.N_S; k.N_L = G.N_L; k.R = G.R; k.L_L = S.L_L; k.L_S = S.L_S; k.S_L = S.S_L; k.n_low = S.n_low;
  k.c = S.c; k.Lact = S.Lact; k.B = G.B;
  k.ola_tx = P.scheme_tx == FC_OLA; k.dtx = S.dtx; k.drx = S.drx; k.lcp = S.lcp; k.soff = S.soff;
  return k;
}

// transform g = (stream s, block or symbol r); the symbol passes also need the
// symbol's low-rate CP and start in the low-rate stream
struct TcCtx {
  int s, r, lcp;
  long long soff;
};

template <int PASS>
__device__ __forceinline__ TcCtx tc_ctx(const TcK& K, int g) {
  constexpr bool sym = PASS == FC_TC_OFDM_MOD || PASS == FC_TC_OFDM_DEMOD;
  const int nT = sym ? K.B : K.R;
  TcCtx c;
  c.s = g / nT;
  c.r = g - c.s * nT;
  c.lcp = 0;
  c.soff = 0;
  if constexpr (sym) {
    c.lcp = __ldg(K.lcp + c.r);
    c.soff = __ldg(K.soff + c.r);
  }
  return c;
}

// signed subcarrier f of bin k and its index in the grid row (or -1): the active
// subcarriers occupy f in [-floor(L_act/2), ceil(L_act/2))
__device__ __forceinline__ int tc_active(int k, int Lact) {
  const int f = k < kN / 2 ? k : k - kN;
  const int lo = Lact / 2;
  return (f >= -lo && f < Lact - lo) ? f + lo : -1;
}

// ---- prologue: where element i of transform c comes from (NULL: zero). The inverse
// passes take the conjugate (IDFT = conj DFT conj), applied when the element is staged.
template <int PASS>
__device__ __forceinline__ const float2* tc_src(const float2* __restrict__ in, const float2* __restrict__ ws,
                                                const TcK& K, const TcCtx& c, int i) {
  if constexpr (PASS == FC_TC_TX_FFT) {       // padded low-rate stream, A window for OLA
    if (K.ola_tx && (i < K.L_L || i >= K.L_L + K.L_S)) return nullptr;
    const long long idx = (long long)c.r * K.L_S + i - K.S_L;
    if (idx < 0 || idx >= K.n_low) return nullptr;
    return ws + (long long)c.s * K.ws_len + K.ws_off + idx;
  } else if constexpr (PASS == FC_TC_RX_FFT) {   // block r of the received frame
    return in + (long long)c.s * K.frame_len + K.offset + (long long)c.r * K.N_S + i;
  } else if constexpr (PASS == FC_TC_OFDM_MOD) { // active subcarriers of symbol r
    const int a = tc_active(i, K.Lact);
    if (a < 0) return nullptr;
    return in + (long long)c.s * K.grid_len + K.grid_off + (long long)c.r * K.Lact + a;
  } else if constexpr (PASS == FC_TC_OFDM_DEMOD) {   // symbol r after its CP in the low-rate stream
    return ws + (long long)c.s * K.ws_len + K.ws_off + c.soff + c.lcp + i;
  } else {                                    // spectrum row
    return ws + (long long)c.s * K.ws_len + K.tc_off + (long long)c.r * kN + i;
  }
}

template <int PASS>
constexpr bool tc_conj_in() {
  return PASS == FC_TC_TX_IFFT || PASS == FC_TC_RX_IFFT || PASS == FC_TC_OFDM_MOD;
}

// 8-byte asynchronous copy global -> shared; src NULL fills zeros (source size 0)
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, const float2* valid_ptr) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src ? src : valid_ptr),
               "r"(src ? 8 : 0)
               : "memory");
}

// The inverse block passes read whole spectrum rows (4096 contiguous samples, 16-byte
// aligned: workspace rows start at even complex offsets): one bulk copy per row,
// completing on an mbarrier. So does the RX block DFT when the received frame keeps its
// blocks 16-byte aligned (tc_rx_rows_aligned). The other passes gather or window:
// per-element copies.
template <int PASS>
constexpr bool tc_bulk() {
  return PASS == FC_TC_TX_IFFT || PASS == FC_TC_RX_IFFT;
}

// block r of stream s starts at in + s frame_len + offset + r N_S: 16-byte aligned for
// every (s, r) when the base is and the three strides are even
__device__ __forceinline__ bool tc_rx_rows_aligned(const float2* in, const TcK& K) {
  return ((uintptr_t)in & 15) == 0 && ((K.frame_len | K.offset | (long long)K.N_S) & 1) == 0;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Bulk form (one thread): both rows of `tile` into stg[t][.] on `bar` (rows past the
// end are not fetched; the staging step zeroes them).
template <int PASS>
__device__ __forceinline__ void tc_prefetch_bulk(float2* stg, const float2* __restrict__ in,
                                                 const float2* __restrict__ ws, const TcK& K, int tile, int total,
                                                 uint64_t* bar) {
  uint32_t bytes = 0;
  for (int t = 0; t < 2; ++t) bytes += (2 * tile + t < total) ? kN * 8u : 0u;
  fence_async_smem();                    // earlier generic reads of stg before the async writes
  mbar_arrive_expect_tx(bar, bytes);
  for (int t = 0; t < 2; ++t) {
    const int g = 2 * tile + t;
    if (g >= total) continue;
    const TcCtx cx = tc_ctx<PASS>(K, g);
    bulk_copy(stg + t * kN, tc_src<PASS>(in, ws, K, cx, 0), kN * 8u, bar);
  }
}

// Stage the raw input of `tile` (two transforms) into stg[t][i]; completes at cp.async.wait_all.
template <int PASS>
__device__ __forceinline__ void tc_prefetch(float2* stg, const float2* __restrict__ in, const float2* __restrict__ ws,
                                            const TcK& K, int tile, int total, int tid) {
#pragma unroll 1
  for (int t = 0; t < 2; ++t) {
    const int g = 2 * tile + t;
    const bool valid = g < total;
    const TcCtx cx = tc_ctx<PASS>(K, valid ? g : 0);
#pragma unroll 4
    for (int j = 0; j < kN / kThreads; ++j) {
      const int i = tid + kThreads * j;
      cp_async8(stg + t * kN + i, valid ? tc_src<PASS>(in, ws, K, cx, i) : nullptr, ws);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// ---- epilogue: bin (or time) k of transform c ----------------------------------------------
template <int PASS>
__device__ __forceinline__ void tc_out(float2* __restrict__ out, float2* __restrict__ ws, const TcK& K, float2 ph,
                                       const TcCtx& c, int k, float2 X) {
  if constexpr (PASS == FC_TC_TX_FFT) {       // shift, D_m (with the scalings), phi_r, bin map (I = 1)
    const float w = __ldg(K.dtx + ((k + kN / 2) & (kN - 1)));
    ws[(long long)c.s * K.ws_len + K.tc_off + (long long)c.r * kN + ((k + K.c) & (kN - 1))] = cscale(cmul(ph, X), w);
  } else if constexpr (PASS == FC_TC_TX_IFFT) {   // y = conj(X); OLA add or OLS S window
    const float2 y = make_float2(X.x, -X.y);
    float2* o = out + (long long)c.s * K.frame_len + K.offset + (long long)c.r * K.N_S + k;
    if (K.ola_tx)
      atomicAdd(o, y);
    else if (k >= K.N_L && k < K.N_L + K.N_S)
      *o = y;
  } else if constexpr (PASS == FC_TC_RX_FFT) {    // gather with conj(phi_r), D_m, inverse shift
    const int kk = (k - K.c) & (kN - 1);
    const float w = __ldg(K.drx + ((kk + kN / 2) & (kN - 1)));
    ws[(long long)c.s * K.ws_len + K.tc_off + (long long)c.r * kN + kk] = cscale(cmulc(X, ph), w);
  } else if constexpr (PASS == FC_TC_OFDM_MOD) {  // time sample k of the symbol, and its CP copy
    const float2 x = make_float2(X.x, -X.y);
    float2* d = ws + (long long)c.s * K.ws_len + K.ws_off + c.soff;
    d[c.lcp + k] = x;
    if (k >= kN - c.lcp) d[k - (kN - c.lcp)] = x;
  } else if constexpr (PASS == FC_TC_OFDM_DEMOD) {   // active bins into the grid row
    const int a = tc_active(k, K.Lact);
    if (a >= 0) out[(long long)c.s * K.grid_len + K.grid_off + (long long)c.r * K.Lact + a] = X;
  } else {                                    // RX_IFFT: OLS keeps [L_L, L_L + L_S) of each block
    if (k < K.L_L || k >= K.L_L + K.L_S) return;
    const long long idx = (long long)c.r * K.L_S + k - K.S_L;
    if (idx >= 0 && idx < K.n_low) ws[(long long)c.s * K.ws_len + K.ws_off + idx] = make_float2(X.x, -X.y);
  }
}

__device__ __forceinline__ void issue_mmas(uint32_t tcol, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo) {
#pragma unroll
  for (int prod = 0; prod < 3; ++prod) {      // hi*hi + hi*lo + lo*hi
    const uint32_t a = prod == 2 ? a_lo : a_hi;
    const uint32_t b = prod == 1 ? b_lo : b_hi;
#pragma unroll
    for (int st = 0; st < 8; ++st) {          // K = 128 in steps of 16 (32 bytes)
      const uint32_t ko = (uint32_t)((st >> 2) * kChunk + (st & 3) * 32);
      mma_f16(tcol, sdesc_kmajor_sw128(a + ko), sdesc_kmajor_sw128(b + ko), kIdesc, prod > 0 || st > 0);
    }
  }
}

template <int PASS>
__global__ void __launch_bounds__(kThreads, 1) k_tc_fc(const TcArgs args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ __align__(8) uint64_t stg_bar;    // bulk staging copies (inverse block passes)
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* b_hi = sm;
  unsigned char* b_lo = sm + kOp;
  unsigned char* a_hi = sm + 2 * kOp;
  unsigned char* a_lo = sm + 3 * kOp;
  float2* stg = reinterpret_cast<float2*>(sm + 4 * kOp);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const FcPlanDev& P = *args.P;
  const TcK K = tc_consts(P);
  const float2* __restrict__ tw = P.sz[P.g[0].size_N].tw;   // W_4096^m
  const float2* __restrict__ twL = P.sz[P.s[0].size_L].tw;
  const float2* __restrict__ g_in = args.in;
  float2* __restrict__ g_out = args.out;
  float2* __restrict__ g_ws = args.ws;

  // DFT-64 operand images into shared memory (already swizzled on the host)
  {
    const uint4* src = reinterpret_cast<const uint4*>(args.dft64);
    uint4* dst = reinterpret_cast<uint4*>(b_hi);
    for (int i = tid; i < 2 * kOp / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init(&stg_bar, 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t sa_hi = smem_u32(a_hi), sa_lo = smem_u32(a_lo), sb_hi = smem_u32(b_hi), sb_lo = smem_u32(b_lo);

  constexpr bool kSym = PASS == FC_TC_OFDM_MOD || PASS == FC_TC_OFDM_DEMOD;
  const int total = args.n_streams * (kSym ? K.B : K.R);
  const int n_tiles = (total + 1) / 2;
  const int q = warp & 3, h = warp >> 2;          // TMEM lane quadrant, column quarter
  const int row = 32 * q + lane;                   // this thread's accumulator row
  const int rt = row >> 6, rlo = row & 63;         // transform in the tile, row within it
  uint32_t phase = 0;
  // twiddles W4096^(n2 k1) of this thread's row n2 = rlo and k1 = 16 h + m: a seed and the
  // step W4096^n2 (both fixed for the kernel), advanced by multiplication (15 steps add
  // at most ~2e-6 relative error)
  const float2 tw_step = __ldg(tw + rlo);
  const float2 tw_seed = __ldg(tw + ((rlo * (16 * h)) & (kN - 1)));

  uint32_t stg_phase = 0;
  // what is in flight, for the exit after a failed wait: a staging copy (completing the
  // stg_bar phase of parity stg_issue) and a GEMM (completing the bar phase mma_issue)
  bool stg_pending = false, mma_pending = false;
  uint32_t stg_issue = 0, mma_issue = 0;
  const bool bulk = tc_bulk<PASS>() || (PASS == FC_TC_RX_FFT && tc_rx_rows_aligned(g_in, K));
  if (blockIdx.x < n_tiles) {
    if (!bulk)
      tc_prefetch<PASS>(stg, g_in, g_ws, K, blockIdx.x, total, tid);
    else if (tid == 0)
      tc_prefetch_bulk<PASS>(stg, g_in, g_ws, K, blockIdx.x, total, &stg_bar);
    stg_pending = true;
    stg_issue = stg_phase;
  }
  // Stage `tile` into A from its staged input (waiting for the copy), then start
  // fetching tile + gridDim.x into the staging buffer. False when a bounded wait gave up.
  auto stage = [&](int tile) -> bool {
    if (!bulk) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      stg_pending = false;
    } else {
      if (mbar_wait(&stg_bar, stg_phase)) {
        stg_pending = false;
      } else {
        atomicExch(args.err, 1);
        abort_flag = 1;
      }
      stg_phase ^= 1;
    }
    __syncthreads();
    if (abort_flag) return false;
    // A1[64 t + n2][(n1, re/im)] = x_t[64 n1 + n2]: each thread converts x_t[64 n1 + n2]
    // for four consecutive n1 = 4 a .. 4 a + 3 of one n2: reads coalesced across the warp
    // (consecutive n2), one 16-byte store per hi/lo
#pragma unroll
    for (int it = 0; it < 2 * kN / 4 / kThreads; ++it) {
      const int e4 = tid + kThreads * it;
      const int t = e4 >> 10, n2 = e4 & 63, a = (e4 >> 6) & 15;
      const bool live = !bulk || 2 * tile + t < total;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 v = live ? stg[t * kN + 64 * (4 * a + j) + n2] : czero();
        if (tc_conj_in<PASS>()) v.y = -v.y;
        split_pack(v, hi[j], lo[j]);
      }
      const uint32_t off = op_off(64 * t + n2, 8 * a);           // 16-byte aligned unit
      *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    fence_async_smem();
    __syncthreads();
    // the staging buffer is free: fetch the tile after this one
    if (tile + (int)gridDim.x < n_tiles) {
      if (!bulk)
        tc_prefetch<PASS>(stg, g_in, g_ws, K, tile + gridDim.x, total, tid);
      else if (tid == 0)
        tc_prefetch_bulk<PASS>(stg, g_in, g_ws, K, tile + gridDim.x, total, &stg_bar);
      stg_pending = true;
      stg_issue = stg_phase;
    }
    return true;
  };
  // one thread issues A x B^T into TMEM columns [col, col + 128)
  auto mma = [&](uint32_t col) {
    if (tid == 0) {
      tc_fence_after();
      issue_mmas(tbase + col, sa_hi, sa_lo, sb_hi, sb_lo);
      mma_commit(&bar);
    }
    mma_pending = true;
    mma_issue = phase;
  };
  // wait for the last issued GEMM; false when the bounded wait gave up. The CTA's first
  // such wait polls at most args.first_wait times (normally the same 2^22 as every other
  // wait; a test sets it to zero to exercise the exit below)
  bool first_wait = true;
  auto wait_mma = [&]() -> bool {
    const uint32_t limit = first_wait ? args.first_wait : (1u << 22);
    first_wait = false;
    if (mbar_wait(&bar, phase, limit)) {
      mma_pending = false;
    } else {
      atomicExch(args.err, 1);
      abort_flag = 1;
    }
    phase ^= 1;
    tc_fence_after();
    __syncthreads();
    return !abort_flag;
  };

  // Per tile: GEMM 1 into columns [0, 128), twiddles back into A, GEMM 2 into columns
  // [128, 256), then the next tile is staged into A and its GEMM 1 issued before this
  // tile's epilogue reads columns [128, 256): the epilogue overlaps the next GEMM 1.
  bool ok = blockIdx.x < n_tiles && stage(blockIdx.x);
  if (ok) mma(0);
  for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
    if (!wait_mma()) break;
    // ---- twiddles; A3[64 t + k1][(n2, re/im)] = A1'[64 t + n2][k1] W4096^(n2 k1) ----------
    // thread: row (t = rt, n2 = rlo), k1 in [16 h, 16 h + 16)
    {
      float d[32];
      tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h), d);
      float2 w = tw_seed;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k1 = 16 * h + m;
        split_store(a_hi, a_lo, op_off(64 * rt + k1, 2 * rlo), cmul(make_float2(d[2 * m], d[2 * m + 1]), w));
        w = cmul(w, tw_step);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    mma(128);
    if (!wait_mma()) break;
    const int next = tile + (int)gridDim.x;
    if (next < n_tiles) {
      if (!stage(next)) break;
      mma(0);
    }
    // ---- epilogue: thread row (t = rt, k1 = rlo), k2 in [16 h, 16 h + 16) ----------------
    const int g = 2 * tile + rt;
    if (g < total) {
      const TcCtx cx = tc_ctx<PASS>(K, g);
      const float2 ph = root_pos_tc(twL, kN, (long long)cx.r * K.c * K.L_S);   // phi_r (L = 4096)
      float d[32];
      tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 + 32 * h), d);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k2 = 16 * h + m;
        tc_out<PASS>(g_out, g_ws, K, ph, cx, rlo + 64 * k2, make_float2(d[2 * m], d[2 * m + 1]));
      }
    }
    tc_fence_before();
    __syncthreads();                       // TMEM columns [128, 256) are free for the next GEMM 2
  }
  if (abort_flag) {
    // a bounded wait gave up: let this CTA's copies and GEMM in flight finish (again with
    // bounded waits) before its shared memory and TMEM are released
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (bulk && stg_pending) mbar_wait(&stg_bar, stg_issue);
    if (mma_pending) mbar_wait(&bar, mma_issue);
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 256);
}

}  // namespace

cudaError_t fc_launch_tc(const FcPlanDev* dP, const unsigned char* dft64, int pass, int n_streams, int n_blocks,
                         const float2* in, float2* out, float2* ws, int* err, int num_sms, cudaStream_t st,
                         unsigned first_wait) {
  TcArgs a{dP, dft64, pass, n_streams, in, out, ws, err, first_wait};
  const int tiles = (n_streams * n_blocks + 1) / 2;
  const int grid = tiles < num_sms ? tiles : num_sms;
  if (grid < 1) return cudaSuccess;
  switch (pass) {
    case FC_TC_TX_FFT: k_tc_fc<FC_TC_TX_FFT><<<grid, kThreads, kSmem, st>>>(a); break;
    case FC_TC_TX_IFFT: k_tc_fc<FC_TC_TX_IFFT><<<grid, kThreads, kSmem, st>>>(a); break;
    case FC_TC_RX_FFT: k_tc_fc<FC_TC_RX_FFT><<<grid, kThreads, kSmem, st>>>(a); break;
    case FC_TC_OFDM_MOD: k_tc_fc<FC_TC_OFDM_MOD><<<grid, kThreads, kSmem, st>>>(a); break;
    case FC_TC_OFDM_DEMOD: k_tc_fc<FC_TC_OFDM_DEMOD><<<grid, kThreads, kSmem, st>>>(a); break;
    default: k_tc_fc<FC_TC_RX_IFFT><<<grid, kThreads, kSmem, st>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t fc_set_tc_smem_limits() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_tc_fc<FC_TC_TX_FFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem))) return e;
  if ((e = cudaFuncSetAttribute(k_tc_fc<FC_TC_TX_IFFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem))) return e;
  if ((e = cudaFuncSetAttribute(k_tc_fc<FC_TC_RX_FFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem))) return e;
  if ((e = cudaFuncSetAttribute(k_tc_fc<FC_TC_OFDM_MOD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem))) return e;
  if ((e = cudaFuncSetAttribute(k_tc_fc<FC_TC_OFDM_DEMOD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)))
    return e;
  return cudaFuncSetAttribute(k_tc_fc<FC_TC_RX_IFFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

// Host image of the DFT-64 B operand (N 128 = (re, im) of output k, K 128 = (re, im) of
// input n): D[row][2k + 0] = Re X[k], D[row][2k + 1] = Im X[k]. Entries from FP64
// cos/sin of 2 pi (n k mod 64) / 64, split into BF16 hi and lo (round to nearest even).
namespace {
uint16_t bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
float bf16_to_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
}  // namespace

void fc_tc_dft64_image(unsigned char* out /* 2 * kOp bytes */) {
  std::memset(out, 0, 2 * kOp);
  const double two_pi = 6.283185307179586476925286766559;
  for (int kk = 0; kk < 64; ++kk)
    for (int nn = 0; nn < 64; ++nn) {
      const double ang = two_pi * (double)((kk * nn) & 63) / 64.0;
      const double cr = std::cos(ang), ci = -std::sin(ang);   // W64^(n k)
      // out re: x_re cr - x_im ci ; out im: x_re ci + x_im cr
      const double v[2][2] = {{cr, -ci}, {ci, cr}};
      for (int co = 0; co < 2; ++co)
        for (int cin = 0; cin < 2; ++cin) {
          const float f = (float)v[co][cin];
          const uint16_t hb = bf16_rne(f);
          const uint16_t lb = bf16_rne((float)((double)v[co][cin] - (double)bf16_to_float(hb)));
          const uint32_t off = op_off(2 * kk + co, 2 * nn + cin);
          std::memcpy(out + off, &hb, 2);
          std::memcpy(out + kOp + off, &lb, 2);
        }
    }
}

size_t fc_tc_dft64_image_bytes() { return 2 * (size_t)kOp; }

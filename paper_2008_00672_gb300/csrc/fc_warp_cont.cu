// Warp-specialised continuous FC kernels (sm_103a) for the 5 MHz NR numerology: one
// subband, short transform L = L_OFDM = 384, long transform N = 512 (I = 4/3), 50 %
// overlap (L_S = 192, N_S = 256), overlap-save on the side the kernel serves.
//
// One warp processes a pair of consecutive FC blocks (eq:BDM, Sec. III-B) or a pair of
// CP-OFDM symbols end to end, with no CTA-wide barrier:
//   * the 384-point transforms of both items run as one four-step FFT of 12 x 32 per
//     item: a 12-point DFT over the 12 values a lane holds (3 x 4 in registers), the
//     twiddles W_384^(lane k1), one transpose through shared memory, and 32-point DFTs
//     in registers on 24 lanes (12 per item; the other 8 lanes idle in that step);
//   * the two 512-point long transforms run as the two-transform four-step FFT of the
//     symbol-synchronized kernels (16 x 32 each);
//   * overlap-save keeps disjoint output ranges, so every sample is written once with a
//     plain store.
// The low-rate CP-OFDM stream sits in the caller's workspace between the OFDM kernels
// and the block kernels (the same layout as the generic continuous kernels).
#include "fc_device.cuh"
#include "fc_internal.cuh"
#include "fc_warp_fft.cuh"

#include <type_traits>

namespace fcdev {

// cos(2 pi m / 24) for m in [0, 24): the exact values of 0..90 degrees in 15-degree
// steps and the quadrant symmetries
__host__ __device__ constexpr float c24_base(int m) {
  return m == 0 ? 1.0f
       : m == 1 ? 0.96592582628906828675f    // cos 15 = (sqrt 6 + sqrt 2) / 4
       : m == 2 ? 0.86602540378443864676f    // cos 30 = sqrt 3 / 2
       : m == 3 ? 0.70710678118654752440f    // cos 45
       : m == 4 ? 0.5f                       // cos 60
       : m == 5 ? 0.25881904510252076235f    // cos 75 = (sqrt 6 - sqrt 2) / 4
                : 0.0f;
}
__host__ __device__ constexpr float c24(int m) {
  return m > 12 ? c24(24 - m) : (m > 6 ? -c24_base(12 - m) : c24_base(m));
}
// sin(2 pi m / 24) = cos(2 pi (m - 6) / 24)
__host__ __device__ constexpr float s24(int m) { return c24((m + 18) % 24); }

// a * W_24^M (forward: exp(-j 2 pi M / 24); inverse: exp(+j 2 pi M / 24))
template <int M, bool INV>
__device__ __forceinline__ float2 tw24(float2 a) {
  constexpr int m = M % 24;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 6) {
    return mul_mj<INV>(a);
  } else if constexpr (m == 12) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (m == 18) {
    return mul_mj<!INV>(a);
  } else {
    constexpr float c = c24(m);
    constexpr float s = s24(m);
    if constexpr (INV) return make_float2(a.x * c - a.y * s, a.y * c + a.x * s);
    else return make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
  }
}

// R = R1 x R2 points (R divides 24), natural order in and out:
//   X[k1 + R1 k2] = sum_t2 W_R2^(t2 k2) W_R^(t2 k1) sum_t1 x[t2 + R2 t1] W_R1^(t1 k1)
template <int R1, int R2, bool INV>
struct DftCT {
  static constexpr int R = R1 * R2;
  template <int T2>
  static __device__ __forceinline__ void inner(const float2* v, float2* a) {
    if constexpr (T2 < R2) {
      float2 t[R1];
#pragma unroll
      for (int t1 = 0; t1 < R1; ++t1) t[t1] = v[T2 + R2 * t1];
      Dft<R1, INV>::run(t);
      twiddle<T2, 0>(t, a);
      inner<T2 + 1>(v, a);
    }
  }
  template <int T2, int K1>
  static __device__ __forceinline__ void twiddle(const float2* t, float2* a) {
    if constexpr (K1 < R1) {
      a[T2 * R1 + K1] = tw24<(T2 * K1 * (24 / R)) % 24, INV>(t[K1]);
      twiddle<T2, K1 + 1>(t, a);
    }
  }
  static __device__ __forceinline__ void run(float2* v) {
    float2 a[R];
    inner<0>(v, a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 t[R2];
#pragma unroll
      for (int t2 = 0; t2 < R2; ++t2) t[t2] = a[t2 * R1 + k1];
      Dft<R2, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
    }
  }
};

template <bool INV>
struct Dft<12, INV> {
  static __device__ __forceinline__ void run(float2* v) { DftCT<3, 4, INV>::run(v); }
};

}  // namespace fcdev

namespace {
using namespace fcdev;
using namespace fcwarp;

constexpr int kWarps = FC_WARP_THREADS / 32;
constexpr int kL = 384, kN = 512, kH = kL / 2;

// Two 384-point DFTs (INV: inverse without 1/n) of one warp, four-step 12 x 32.
// In: lane l holds x_b[32 a + l] in v[12 b + a] (a < 12, b < 2).
// Out: lane 12 b + k1 (< 24) holds X_b[k1 + 12 k2] in v[k2]; lanes 24..31 hold nothing.
// scr: the warp's transpose buffer (32 x kPad float2); tw = forward table of size 384,
// or with STAGED a per-lane step table in shared memory (row k1 holds W_384^(k1 lane)).
template <bool INV, bool STAGED = false>
__device__ __forceinline__ void dft384x2(float2 (&v)[32], float2* scr, const float2* __restrict__ tw, int lane) {
  Dft<12, INV>::run(v);
  Dft<12, INV>::run(v + 12);
#pragma unroll
  for (int k1 = 1; k1 < 12; ++k1) {              // W_384^(lane k1), the same for both items
    float2 w = STAGED ? tw[k1 * 32 + lane] : __ldg(tw + lane * k1);
    if (INV) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
    v[12 + k1] = cmul(v[12 + k1], w);
  }
#pragma unroll
  for (int i = 0; i < 24; ++i) scr[i * kPad + lane] = v[i];
  __syncwarp();
#pragma unroll
  for (int n = 0; n < 32; ++n) v[n] = scr[lane * kPad + n];   // rows 24..31: unused values
  __syncwarp();
  Dft<32, INV>::run(v);
}

__device__ __forceinline__ int signed_bin384(int k) { return k < kH ? k : k - kL; }

// The block kernels' tables staged in shared memory once per CTA, after the warps'
// transpose buffers: per-lane step twiddles (row e holds W^(e lane), lane = 0..31; one
// conflict-free read per twiddle) of the 384-point four-step (12 rows) and of the
// two 512-point transforms (16 rows), then the subband's weights (TX or RX), which the bin
// loops read at positions that depend on the carrier.
constexpr int kContTables = 12 * 32 + 16 * 32;       // float2, then kL floats of weights
constexpr size_t kContTableBytes = kContTables * sizeof(float2) + kL * sizeof(float);

struct ContTables {
  const float2* twL;      // per-lane step table, 384 points
  const float2* twN;      // per-lane step table, 512 points
  const float* w;
};

__device__ __forceinline__ ContTables stage_cont_tables(const FcPlanDev& P, float2* base, const float* weights) {
  const FcSubDev& S = P.s[0];
  const FcGroupDev& G = P.g[0];
  float* w = reinterpret_cast<float*>(base + kContTables);
  stage_lane_twiddles(base, P.sz[S.size_L].tw, kL, 12);
  stage_lane_twiddles(base + 12 * 32, P.sz[G.size_N].tw, kN, 16);
  for (int m = threadIdx.x; m < kL; m += blockDim.x) w[m] = __ldg(weights + m);
  __syncthreads();
  return ContTables{base, base + 12 * 32, w};
}

// warp-level persistent item loop: items [0, total), warp w of the grid takes w, w + W, ...
struct WarpItems {
  long long first, step;
  __device__ WarpItems() {
    first = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    step = (long long)gridDim.x * kWarps;
  }
};

// ---------------------------------------------------------------------------
// T1-T2: OFDM IDFT and CP insertion of symbols 2p, 2p + 1 into the low-rate stream
// ---------------------------------------------------------------------------
template <typename TI>
__global__ void __launch_bounds__(FC_WARP_THREADS, FC_WARP_CONT_MIN_BLOCKS)
k_ofdm_mod_w384(const FcPlanDev* __restrict__ gP, int n_streams, const TI* __restrict__ grid,
                float2* __restrict__ ws) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) float2 wscr[];
  pdl_trigger();                                    // the block kernel may stage its tables meanwhile
  load_plan_w(P, gP);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kTrans;
  const FcSubDev& S = P.s[0];
  const int B = P.g[0].B, pairs = (B + 1) / 2;
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  const float2* __restrict__ twL = P.sz[S.size_L].tw;
  const long long total = (long long)n_streams * pairs;
  for (long long item = WarpItems().first; item < total; item += WarpItems().step) {
    const int stream = (int)(item / pairs), n0 = 2 * (int)(item - (long long)stream * pairs);
    const TI* __restrict__ rows = grid + (size_t)stream * P.grid_len + S.grid_off;
    float2 v[32];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const bool live = n0 + b < B;
#pragma unroll
      for (int a = 0; a < 12; ++a) {
        const int f = signed_bin384(32 * a + lane);
        v[12 * b + a] = (live && f >= -hl && f < hu) ? ld_io(rows + (long long)(n0 + b) * S.Lact + f + hl) : czero();
      }
    }
#pragma unroll
    for (int a = 24; a < 32; ++a) v[a] = czero();
    dft384x2<true>(v, scr, twL, lane);
    // K_{L_CP} (eq:TX_CPins): body sample t at L_CP + t, and the last L_CP samples again in front
    if (lane < 24) {
      const int b = lane >= 12, k1 = lane - 12 * b, n = n0 + b;
      if (n < B) {
        const int lcp = S.lcp[n];
        float2* dst = ws + (size_t)stream * P.ws_len + S.ws_off + S.soff[n];
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int t = k1 + 12 * k2;
          dst[lcp + t] = v[k2];
          if (t >= kL - lcp) dst[t - (kL - lcp)] = v[k2];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// T3-T7, overlap-save: FC blocks 2p, 2p + 1 of the low-rate stream -> waveform
// ---------------------------------------------------------------------------
template <typename TO>
__global__ void __launch_bounds__(FC_WARP_THREADS, FC_WARP_CONT_MIN_BLOCKS)
k_tx_cont_w384(const FcPlanDev* __restrict__ gP, int n_streams, const float2* __restrict__ ws,
               TO* __restrict__ wave) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) float2 wscr[];
  load_plan_w(P, gP);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kTrans;   // transposes, and the spectra between them
  const FcGroupDev& G = P.g[0];
  const FcSubDev& S = P.s[0];
  const int R = G.R, pairs = (R + 1) / 2;
  const ContTables T = stage_cont_tables(P, wscr + kWarps * kTrans, S.dtx);
  pdl_wait();                                       // the low-rate stream of the OFDM kernel
  const long long total = (long long)n_streams * pairs;
  for (long long item = WarpItems().first; item < total; item += WarpItems().step) {
    const int stream = (int)(item / pairs), r0 = 2 * (int)(item - (long long)stream * pairs);
    const int nb = R - r0 < 2 ? R - r0 : 2;
    const float2* __restrict__ s = ws + (size_t)stream * P.ws_len + S.ws_off;
    float2 v[32];
    // T3: block r = r0 + b is [r L_S - S_L, r L_S - S_L + L) of the zero-padded stream
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
      for (int a = 0; a < 12; ++a) {
        const int pos = (r0 + b) * S.L_S + 32 * a + lane - S.S_L;
        v[12 * b + a] = (b < nb && pos >= 0 && pos < S.n_low) ? __ldg(s + pos) : czero();
      }
    }
#pragma unroll
    for (int a = 24; a < 32; ++a) v[a] = czero();
    // T4: short DFTs
    dft384x2<false, true>(v, scr, T.twL, lane);
    // T5: shift P^(L/2), D_m and phi_r, bin map into the two 512-bin spectra
    float2* map = scr;
#pragma unroll
    for (int a = 0; a < 32; ++a) map[32 * a + lane] = czero();
    __syncwarp();
    if (lane < 24) {
      const int b = lane >= 12, k1 = lane - 12 * b;
      if (b < nb) {
        const float2 ph = root_pos(P.sz[G.size_N].tw, kN, (long long)S.c * (r0 + b) * G.N_S);
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int k = k1 + 12 * k2;
          int p = k + kH;
          if (p >= kL) p -= kL;
          if (p >= S.p_lo && p < S.p_hi)
            map[kN * b + ((S.c + p - kH) & (kN - 1))] = cscale(cmul(v[k2], ph), T.w[p]);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 16; ++a) v[16 * b + a] = map[kN * b + 32 * a + lane];
    __syncwarp();
    // T6: long IDFTs (1/N and sqrt(I) folded into D); step twiddles from the global table
    // (measured faster here than the staged per-lane table, which the RX kernel uses)
    conj32(v);
    warp_fft(v, scr, P.sz[G.size_N].tw, P.sz[G.size_N].tw, lane, true);
    conj32(v);
    // T7: S window [N_L, N_L + N_S) of block r at r N_S; the frame's first N_L and last
    // N_T samples, which no window covers, are zeros
    const int b = lane >> 4, k1 = lane & 15;
    if (b < nb) {
      const int r = r0 + b;
      TO* __restrict__ out = wave + (size_t)stream * P.frame_len + (long long)r * G.N_S;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int tau = k1 + 16 * k2;
        const bool keep = tau >= G.N_L && tau < G.N_L + G.N_S;
        if (keep) st_io(out + tau, v[k2]);
        else if ((r == 0 && tau < G.N_L) || (r == R - 1 && tau >= G.N_L + G.N_S)) st_io(out + tau, czero());
      }
    }
  }
}

// ---------------------------------------------------------------------------
// R1-R5, overlap-save: FC blocks 2p, 2p + 1 of the waveform -> low-rate stream
// ---------------------------------------------------------------------------
template <typename TI>
__global__ void __launch_bounds__(FC_WARP_THREADS, FC_WARP_CONT_MIN_BLOCKS)
k_rx_cont_w384(const FcPlanDev* __restrict__ gP, int n_streams, const TI* __restrict__ wave,
               float2* __restrict__ ws) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) float2 wscr[];
  pdl_trigger();                                    // the OFDM kernel may start meanwhile
  load_plan_w(P, gP);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kTrans;
  const FcGroupDev& G = P.g[0];
  const FcSubDev& S = P.s[0];
  const int R = G.R, pairs = (R + 1) / 2;
  const ContTables T = stage_cont_tables(P, wscr + kWarps * kTrans, S.drx);
  const long long total = (long long)n_streams * pairs;
  for (long long item = WarpItems().first; item < total; item += WarpItems().step) {
    const int stream = (int)(item / pairs), r0 = 2 * (int)(item - (long long)stream * pairs);
    const int nb = R - r0 < 2 ? R - r0 : 2;
    const TI* __restrict__ x = wave + (size_t)stream * P.frame_len;
    float2 v[32];
    // R1: block r is the N samples from r N_S (overlap-save: no window)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 16; ++a)
        v[16 * b + a] = b < nb ? ld_io(x + (long long)(r0 + b) * G.N_S + 32 * a + lane) : czero();
    // R2: long DFTs; lane k1 + 16 T holds Y_T[k1 + 16 k2] in v[k2]
    warp_fft<true>(v, scr, T.twN, T.twN, lane, true);
    float2* map = scr;
    {
      const int half = lane >> 4, k1 = lane & 15;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) map[kN * half + k1 + 16 * k2] = v[k2];
    }
    __syncwarp();
    // R3: gather with conj(phi_r), D_m, inverse shift, into the short IDFTs' input layout
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float2 ph = root_pos(P.sz[G.size_N].tw, kN, (long long)S.c * (r0 + b) * G.N_S);
#pragma unroll
      for (int a = 0; a < 12; ++a) {
        const int k = 32 * a + lane;
        int p = k + kH;
        if (p >= kL) p -= kL;
        float2 u = czero();
        if (b < nb && p >= S.p_lo && p < S.p_hi)
          u = cscale(cmulc(map[kN * b + ((S.c + p - kH) & (kN - 1))], ph), T.w[p]);
        v[12 * b + a] = u;
      }
    }
#pragma unroll
    for (int a = 24; a < 32; ++a) v[a] = czero();
    __syncwarp();
    // R4: short IDFTs
    dft384x2<true, true>(v, scr, T.twL, lane);
    // R5: keep [L_L, L_L + L_S) of block r at low-rate position r L_S + L_L - S_L
    if (lane < 24) {
      const int b = lane >= 12, k1 = lane - 12 * b;
      if (b < nb) {
        float2* __restrict__ d = ws + (size_t)stream * P.ws_len + S.ws_off;
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int t = k1 + 12 * k2;
          const int pos = (r0 + b) * S.L_S + t - S.S_L;
          if (t >= S.L_L && t < S.L_L + S.L_S && pos >= 0 && pos < S.n_low) d[pos] = v[k2];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// R5-R6: CP removal and OFDM DFT of symbols 2p, 2p + 1, active bins to the grid
// ---------------------------------------------------------------------------
template <typename TO>
__global__ void __launch_bounds__(FC_WARP_THREADS, FC_WARP_CONT_MIN_BLOCKS)
k_ofdm_demod_w384(const FcPlanDev* __restrict__ gP, int n_streams, const float2* __restrict__ ws,
                  TO* __restrict__ grid) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) float2 wscr[];
  load_plan_w(P, gP);
  __syncthreads();
  pdl_wait();                                       // the low-rate stream of the block kernel
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kTrans;
  const FcSubDev& S = P.s[0];
  const int B = P.g[0].B, pairs = (B + 1) / 2;
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  const float2* __restrict__ twL = P.sz[S.size_L].tw;
  const long long total = (long long)n_streams * pairs;
  for (long long item = WarpItems().first; item < total; item += WarpItems().step) {
    const int stream = (int)(item / pairs), n0 = 2 * (int)(item - (long long)stream * pairs);
    const float2* __restrict__ s = ws + (size_t)stream * P.ws_len + S.ws_off;
    float2 v[32];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int n = n0 + b;
      const float2* __restrict__ body = s + (n < B ? S.soff[n] + S.lcp[n] : 0);
#pragma unroll
      for (int a = 0; a < 12; ++a) v[12 * b + a] = n < B ? __ldg(body + 32 * a + lane) : czero();
    }
#pragma unroll
    for (int a = 24; a < 32; ++a) v[a] = czero();
    dft384x2<false>(v, scr, twL, lane);
    if (lane < 24) {
      const int b = lane >= 12, k1 = lane - 12 * b, n = n0 + b;
      if (n < B) {
        TO* __restrict__ row = grid + (size_t)stream * P.grid_len + S.grid_off + (long long)n * S.Lact;
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int f = signed_bin384(k1 + 12 * k2);
          if (f >= -hl && f < hu) st_io(row + f + hl, v[k2]);
        }
      }
    }
  }
}

// pdl: a programmatic dependent of the call's first kernel (which triggers at its start;
// the dependent waits before it reads the workspace)
template <class K, class TI, class TO>
cudaError_t launch_w(K kern, long long items, int num_sms, cudaStream_t st, const FcPlanDev* dP, int n_streams,
                     const TI* in, TO* out, size_t tables = 0, bool pdl = false) {
  const size_t smem = (size_t)kWarps * kTrans * sizeof(float2) + tables;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FC_WARP_THREADS, smem);
  if (e != cudaSuccess) return e;
  long long ctas = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
  const long long need = (items + kWarps - 1) / kWarps;
  if (ctas > need) ctas = need;
  if (ctas < 1) return cudaSuccess;
  return fcwarp::launch_k(kern, (unsigned)ctas, FC_WARP_THREADS, smem, st, pdl, dP, n_streams, in, out);
}

}  // namespace

// io: FC_IO_* bits (complex-BF16 grid / waveform; the workspace stays complex64)
cudaError_t fc_launch_tx_cont_warp(const FcPlanDev* dP, int n_streams, int n_symbols, int n_blocks, const void* grid,
                                   float2* ws, void* wave, int io, int num_sms, cudaStream_t st) {
  const long long syms = (long long)n_streams * ((n_symbols + 1) / 2), blks = (long long)n_streams * ((n_blocks + 1) / 2);
  cudaError_t e = (io & FC_IO_IN_BF16)
                      ? launch_w(k_ofdm_mod_w384<bf2>, syms, num_sms, st, dP, n_streams, (const bf2*)grid, ws)
                      : launch_w(k_ofdm_mod_w384<float2>, syms, num_sms, st, dP, n_streams, (const float2*)grid, ws);
  if (e != cudaSuccess) return e;
  return (io & FC_IO_OUT_BF16)
             ? launch_w(k_tx_cont_w384<bf2>, blks, num_sms, st, dP, n_streams, (const float2*)ws, (bf2*)wave,
                        kContTableBytes, true)
             : launch_w(k_tx_cont_w384<float2>, blks, num_sms, st, dP, n_streams, (const float2*)ws, (float2*)wave,
                        kContTableBytes, true);
}

cudaError_t fc_launch_rx_cont_warp(const FcPlanDev* dP, int n_streams, int n_symbols, int n_blocks, const void* wave,
                                   float2* ws, void* grid, int io, int num_sms, cudaStream_t st) {
  const long long syms = (long long)n_streams * ((n_symbols + 1) / 2), blks = (long long)n_streams * ((n_blocks + 1) / 2);
  cudaError_t e = (io & FC_IO_IN_BF16)
                      ? launch_w(k_rx_cont_w384<bf2>, blks, num_sms, st, dP, n_streams, (const bf2*)wave, ws,
                                 kContTableBytes)
                      : launch_w(k_rx_cont_w384<float2>, blks, num_sms, st, dP, n_streams, (const float2*)wave, ws,
                                 kContTableBytes);
  if (e != cudaSuccess) return e;
  return (io & FC_IO_OUT_BF16)
             ? launch_w(k_ofdm_demod_w384<bf2>, syms, num_sms, st, dP, n_streams, (const float2*)ws, (bf2*)grid, 0,
                        true)
             : launch_w(k_ofdm_demod_w384<float2>, syms, num_sms, st, dP, n_streams, (const float2*)ws, (float2*)grid, 0,
                        true);
}

// Warp-centric symbol-synchronized FC kernels (sm_103a) for the numerologies
// with I = N/L = 2 and L in {512, 1024} (one subband per numerology group).
//
// One warp processes one symbol job (Sec. III-C for TX, Sec. IV for RX) end to
// end with no CTA-wide barrier:
//   * 1024-point transforms are four-step 32 x 32 FFTs held in registers
//     (32 values per lane) with one shared-memory transpose; two 512-point
//     transforms run together as 16 x 32 four-step FFTs;
//   * the long N = 2048 transform is split by one radix-2 step into two
//     1024-point transforms (even and odd output samples for the TX IDFT,
//     even and odd bins for the RX DFT);
//   * the segmentation of the zero-padded symbol into the two FC blocks
//     (eq:padding, R_L^{(r)}) is a register renaming, because L/4 and L/2 are
//     multiples of the 32-sample stride of the register layout;
//   * TX overlap-add (blocks of a symbol, neighbouring symbols, numerology
//     groups; eq:multi-symb) is done with vector reductions into the zeroed
//     output waveform, so warps never wait for each other.
#include "fc_device.cuh"
#include "fc_internal.cuh"

namespace {
using namespace fcdev;

constexpr int kPad = 33;                       // transpose row stride in float2
constexpr int kTrans = 32 * kPad;              // per-warp transpose buffer (float2)
constexpr int kMap = 1024;                     // per-warp spectrum / re-layout buffer (float2)
constexpr int kScratch = kTrans + kMap;
constexpr int kWarps = FC_WARP_THREADS / 32;

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

// v[k] *= W_n^{+-lane k} for k = 1..K-1, with W^{lane k} = W^{4 m lane} W^{j lane} (k = 4 m + j):
// K/4 + 3 table loads and one complex multiply per twiddle (one rounding away from the table).
template <int K, bool INV>
__device__ __forceinline__ void step_twiddles(float2* v, const float2* __restrict__ tw, int lane) {
  float2 tj[4];
  tj[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int j = 1; j < 4; ++j) tj[j] = __ldg(tw + lane * j);
#pragma unroll
  for (int m = 0; m < K / 4; ++m) {
    const float2 tm = m ? __ldg(tw + lane * 4 * m) : make_float2(1.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * m + j;
      if (k == 0) continue;
      float2 w = (m == 0) ? tj[j] : (j == 0 ? tm : cmul(tm, tj[j]));
      if (INV) w.y = -w.y;
      v[k] = cmul(v[k], w);
    }
  }
}

// Four-step 1024-point FFT. In: lane b holds x[32 a + b] in v[a].
// Out: lane k1 holds X[k1 + 32 k2] in v[k2]. tw = forward table of size 1024.
template <bool INV>
__device__ __forceinline__ void warp_fft1024(float2 (&v)[32], float2* scr, const float2* __restrict__ tw, int lane) {
  Dft<32, INV>::run(v);
  step_twiddles<32, INV>(v, tw, lane);
#pragma unroll
  for (int k = 0; k < 32; ++k) scr[k * kPad + lane] = v[k];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < 32; ++b) v[b] = scr[lane * kPad + b];
  __syncwarp();
  Dft<32, INV>::run(v);
}

// Two four-step 512-point FFTs (16 x 32). In: lane b holds x_T[32 a + b] in
// v[16 T + a], a < 16. Out: lane L = k1 + 16 T holds X_T[k1 + 16 k2] in v[k2].
// tw = forward table of size 512.
template <bool INV>
__device__ __forceinline__ void warp_fft512x2(float2 (&v)[32], float2* scr, const float2* __restrict__ tw, int lane) {
  Dft<16, INV>::run(v);
  Dft<16, INV>::run(v + 16);
  {
    float2 t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t[k] = make_float2(1.f, 0.f);
    step_twiddles<16, INV>(t, tw, lane);       // t[k] = W_512^{+-lane k}
#pragma unroll
    for (int k = 1; k < 16; ++k) {
      v[k] = cmul(v[k], t[k]);
      v[16 + k] = cmul(v[16 + k], t[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) scr[k * kPad + lane] = v[k];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < 32; ++b) v[b] = scr[lane * kPad + b];
  __syncwarp();
  Dft<32, INV>::run(v);
}

__device__ __forceinline__ float weight(const FcSubDev& S, const float* __restrict__ d, int p) {
  return (p >= S.p_lo && p < S.p_hi) ? __ldg(d + p) : 0.f;
}

// ---------------------------------------------------------------------------
// TX, L = 1024, N = 2048
// ---------------------------------------------------------------------------
__device__ __noinline__ void tx_job_1024(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                            const float2* __restrict__ gsrc, float2* __restrict__ wdst, float2* scr,
                                            float2* map, int lane) {
  constexpr int L = 1024;
  const float2* __restrict__ twL = P.sz[S.size_L].tw;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const int n = jb.index;
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  const float2* __restrict__ row = gsrc + S.grid_off + (long long)n * S.Lact;
  float2 v[32];
  // T1: active subcarriers into the inverse-transform layout (bin 32 a + lane)
#pragma unroll
  for (int a = 0; a < 32; ++a) {
    const int i = 32 * a + lane;
    const int f = i < L / 2 ? i : i - L;
    v[a] = (f >= -hl && f < hu) ? __ldg(row + f + hl) : czero();
  }
  warp_fft1024<true>(v, scr, twL, lane);          // body[k1 + 32 k2] in lane k1, v[k2]
  float2 bd[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) bd[k] = v[k];
  const int lcp = S.lcp[n], ncp = G.ncp[n];
  const bool ols = P.scheme_tx == FC_OLS;
  const bool v4 = ((jb.start & 1) == 0);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    // T2-T3: block r of the padded symbol: position t = 32 a + lane holds body[(t - L/4 + r L/2) mod L]
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      const int t = 32 * a + lane;
      bool keep;
      if (!ols) keep = (r == 0) ? (t >= L / 4 - lcp && t < 3 * L / 4) : (t >= L / 4 && t < 3 * L / 4);
      else keep = (r == 0) ? (t >= L / 4 - lcp) : (t < 3 * L / 4);
      v[a] = keep ? bd[(a + 24 + 16 * r) & 31] : czero();
    }
    // T4: short DFT
    warp_fft1024<false>(v, scr, twL, lane);       // U[k1 + 32 k2]
    // T5: shift, D_m, bin map with phi_r theta_n; the 1024-bin band folds one-to-one onto q mod 1024
    const float2 ph = root_pos(twN, 2048, (long long)S.c * (G.cps[n] + r * G.N_S));
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int k = lane + 32 * k2;
      const int kt = k < L / 2 ? k : k - L;
      const float w = weight(S, S.dtx, kt + L / 2);
      map[(S.c + kt) & 1023] = cscale(cmul(v[k2], ph), w);
    }
    __syncwarp();
    // T6: long IDFT as two 1024-point IDFTs of the folded spectrum (even / odd output samples)
    float2 u[32], x[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      const int qp = 32 * a + lane;
      int kt = (qp - S.c) & 1023;
      if (kt >= 512) kt -= 1024;
      const float2 y = map[qp];
      u[a] = y;
      x[a] = cmulc(y, __ldg(twN + ((S.c + kt) & 2047)));    // y * exp(+j 2 pi q / 2048)
    }
    __syncwarp();
    warp_fft1024<true>(u, scr, twL, lane);        // output sample 2 (k1 + 32 k2)
    warp_fft1024<true>(x, scr, twL, lane);        // output sample 2 (k1 + 32 k2) + 1
    // T7: OLS window, R_N^{(r)} and Gamma_sigma placement by reduction into the waveform
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int tau = 2 * (lane + 32 * k2);
      float2 a0 = u[k2], a1 = x[k2];
      if (ols) {
        const int lo = (r == 0) ? G.N_L - ncp : G.N_L, hi = G.N_L + G.N_S;
        if (!(tau >= lo && tau < hi)) a0 = czero();
        if (!(tau + 1 >= lo && tau + 1 < hi)) a1 = czero();
      }
      float2* dst = wdst + jb.start + r * (2048 / 2) + tau;
      if (v4) {
        atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a0.x, a0.y, a1.x, a1.y));
      } else {
        atomicAdd(dst, a0);
        atomicAdd(dst + 1, a1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// TX, L = 512, N = 1024
// ---------------------------------------------------------------------------
__device__ __noinline__ void tx_job_512(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                           const float2* __restrict__ gsrc, float2* __restrict__ wdst, float2* scr,
                                           float2* map, int lane) {
  constexpr int L = 512;
  const float2* __restrict__ twL = P.sz[S.size_L].tw;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const int n = jb.index;
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  const float2* __restrict__ row = gsrc + S.grid_off + (long long)n * S.Lact;
  float2 v[32];
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    const int i = 32 * a + lane;
    const int f = i < L / 2 ? i : i - L;
    v[a] = (f >= -hl && f < hu) ? __ldg(row + f + hl) : czero();
    v[16 + a] = czero();
  }
  warp_fft512x2<true>(v, scr, twL, lane);         // lanes 0..15: body[k1 + 16 k2] in v[k2]
  if (lane < 16) {
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) map[lane + 16 * k2] = v[k2];
  }
  __syncwarp();
  const int lcp = S.lcp[n], ncp = G.ncp[n];
  const bool ols = P.scheme_tx == FC_OLS;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      const int t = 32 * a + lane;
      bool keep;
      if (!ols) keep = (r == 0) ? (t >= L / 4 - lcp && t < 3 * L / 4) : (t >= L / 4 && t < 3 * L / 4);
      else keep = (r == 0) ? (t >= L / 4 - lcp) : (t < 3 * L / 4);
      v[16 * r + a] = keep ? map[(t - L / 4 + r * (L / 2)) & (L - 1)] : czero();
    }
  }
  __syncwarp();
  warp_fft512x2<false>(v, scr, twL, lane);        // lane k1 + 16 r: U_r[k1 + 16 k2] in v[k2]
  const int myr = lane >> 4, k1 = lane & 15;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int a = 0; a < 32; ++a) map[32 * a + lane] = czero();
    __syncwarp();
    if (myr == r) {
      const float2 ph = root_pos(twN, 1024, (long long)S.c * (G.cps[n] + r * G.N_S));
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int k = k1 + 16 * k2;
        const int kt = k < L / 2 ? k : k - L;
        const float w = weight(S, S.dtx, kt + L / 2);
        map[(S.c + kt) & 1023] = cscale(cmul(v[k2], ph), w);
      }
    }
    __syncwarp();
    float2 u[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) u[a] = map[32 * a + lane];
    __syncwarp();
    warp_fft1024<true>(u, scr, twN, lane);        // sample k1' + 32 k2 of block r
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int tau = lane + 32 * k2;
      float2 a0 = u[k2];
      if (ols) {
        const int lo = (r == 0) ? G.N_L - ncp : G.N_L, hi = G.N_L + G.N_S;
        if (!(tau >= lo && tau < hi)) a0 = czero();
      }
      atomicAdd(wdst + jb.start + r * (1024 / 2) + tau, a0);
    }
  }
}

// ---------------------------------------------------------------------------
// RX, N = 2048, L = 1024
// ---------------------------------------------------------------------------
__device__ __noinline__ void rx_job_1024(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                            const float2* __restrict__ src, float2* __restrict__ gdst, float2* scr,
                                            float2* map, int lane) {
  constexpr int L = 1024;
  const float2* __restrict__ twL = P.sz[S.size_L].tw;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const int n = jb.index;
  const bool ola = P.scheme_rx == FC_OLA;
  float2 h[32];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    // R1-R2: block r, radix-2 split of the 2048-point DFT into even and odd bins
    const float2* __restrict__ x = src + jb.start + r * (2048 / 2);
    float2 u[32], w[32];
    // R3: gather the subband's 1024 bins with conj(phi_r theta_n), D_m, inverse shift; the even
    // bins right after their transform, so only one half-spectrum is live in registers
    const float2 ph = root_pos(twN, 2048, (long long)S.c * (G.cps[n] + r * G.N_S));
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float2 (&X)[32] = s ? w : u;
      // even bins: DFT of x0 + x1; odd bins: DFT of (x0 - x1) exp(-j 2 pi tp / 2048)
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        const int tp = 32 * a + lane;
        float2 x0 = __ldg(x + tp), x1 = __ldg(x + tp + 1024);
        if (ola) {                                 // A window [N_L, N_L + N_S) = [512, 1536)
          if (tp < 512) x0 = czero();
          if (tp >= 512) x1 = czero();
        }
        X[a] = s ? cmul(csub(x0, x1), __ldg(twN + tp)) : cadd(x0, x1);
      }
      warp_fft1024<false>(X, scr, twL, lane);     // bin 2 (k1 + 32 k2) + s
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int q = 2 * (lane + 32 * k2) + s;
        int kt = (q - S.c) & 2047;
        if (kt >= 1024) kt -= 2048;
        if (kt >= -L / 2 && kt < L / 2) {
          const float wt = weight(S, S.drx, kt + L / 2);
          map[kt & (L - 1)] = cscale(cmulc(X[k2], ph), wt);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 32; ++a) u[a] = map[32 * a + lane];
    __syncwarp();
    // R4: short IDFT
    warp_fft1024<true>(u, scr, twL, lane);        // z_r[k1 + 32 k2] in u[k2]
    // R5: S window + concatenation (eq:concat2), or OLA of both blocks; x_ofdm[t], t = lane + 32 k2
    if (!ola) {
#pragma unroll
      for (int j = 0; j < 16; ++j) h[16 * r + j] = u[j + 8];
    } else {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (r == 0) h[k] = (k < 24) ? u[k + 8] : czero();
        else if (k >= 8) h[k] = cadd(h[k], u[k - 8]);
      }
    }
  }
  // R6: OFDM demodulation and active-bin output
  warp_fft1024<false>(h, scr, twL, lane);
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  float2* __restrict__ row = gdst + S.grid_off + (long long)n * S.Lact;
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const int bin = lane + 32 * k2;
    const int f = bin < L / 2 ? bin : bin - L;
    if (f >= -hl && f < hu) row[f + hl] = h[k2];
  }
}

// ---------------------------------------------------------------------------
// RX, N = 1024, L = 512
// ---------------------------------------------------------------------------
__device__ __noinline__ void rx_job_512(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                           const float2* __restrict__ src, float2* __restrict__ gdst, float2* scr,
                                           float2* map, int lane) {
  constexpr int L = 512;
  const float2* __restrict__ twL = P.sz[S.size_L].tw;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const int n = jb.index;
  const bool ola = P.scheme_rx == FC_OLA;
  float2 X0[32], X1[32];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float2* __restrict__ x = src + jb.start + r * (1024 / 2);
    float2 (&u)[32] = r ? X1 : X0;
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      const int t = 32 * a + lane;
      float2 xv = __ldg(x + t);
      if (ola && !(t >= G.N_L && t < G.N_L + G.N_S)) xv = czero();
      u[a] = xv;
    }
    warp_fft1024<false>(u, scr, twN, lane);       // bin k1 + 32 k2
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float2 ph = root_pos(twN, 1024, (long long)S.c * (G.cps[n] + r * G.N_S));
    const float2 (&u)[32] = r ? X1 : X0;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int q = lane + 32 * k2;
      int kt = (q - S.c) & 1023;
      if (kt >= 512) kt -= 1024;
      if (kt >= -L / 2 && kt < L / 2) {
        const float wt = weight(S, S.drx, kt + L / 2);
        map[r * L + (kt & (L - 1))] = cscale(cmulc(u[k2], ph), wt);
      }
    }
  }
  __syncwarp();
  float2 v[32];
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    v[a] = map[32 * a + lane];
    v[16 + a] = map[L + 32 * a + lane];
  }
  __syncwarp();
  warp_fft512x2<true>(v, scr, twL, lane);         // lane k1 + 16 r: z_r[k1 + 16 k2]
  {
    const int r = lane >> 4, k1 = lane & 15;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) map[r * L + k1 + 16 * k2] = v[k2];
  }
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    const int t = 32 * a + lane;
    float2 val;
    if (!ola) {
      val = t < L / 2 ? map[L / 4 + t] : map[L + t - L / 4];
    } else {
      val = czero();
      if (L / 4 + t < L) val = map[L / 4 + t];
      if (t >= L / 4) val = cadd(val, map[L + t - L / 4]);
    }
    v[a] = val;
    v[16 + a] = czero();
  }
  __syncwarp();
  warp_fft512x2<false>(v, scr, twL, lane);        // lanes 0..15: X[k1 + 16 k2]
  if (lane < 16) {
    const int hl = S.Lact / 2, hu = S.Lact - hl;
    float2* __restrict__ row = gdst + S.grid_off + (long long)n * S.Lact;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int bin = lane + 16 * k2;
      const int f = bin < L / 2 ? bin : bin - L;
      if (f >= -hl && f < hu) row[f + hl] = v[k2];
    }
  }
}

// ---------------------------------------------------------------------------
// kernels: one CTA per (stream, chunk), warps take jobs from a shared counter
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(FC_WARP_THREADS, 3)
k_tx_sync_warp(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, const FcChunk* __restrict__ chunks,
               int n_chunks, int zero_output, const float2* __restrict__ grid, float2* __restrict__ wave) {
  __shared__ FcPlanDev P;
  __shared__ int next_job;
  extern __shared__ __align__(16) float2 wscr[];
  load_plan_w(P, gP);
  const int stream = blockIdx.x / n_chunks;
  const FcChunk ch = chunks[blockIdx.x - stream * n_chunks];
  if (threadIdx.x == 0) next_job = ch.j0;
  __syncthreads();                                  // the plan copy is complete before any use
  const float2* gsrc = grid + (size_t)stream * P.grid_len;
  float2* wdst = wave + (size_t)stream * P.frame_len;
  if (zero_output) {   // the CTA owns the whole stream: clear it before the reductions
    for (int i = threadIdx.x; i < P.frame_len; i += blockDim.x) wdst[i] = czero();
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kScratch;
  float2* map = scr + kTrans;
  while (true) {
    int j = 0;
    if (lane == 0) j = atomicAdd(&next_job, 1);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= ch.j1) break;
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    const FcSubDev& S = P.s[G.first_sub];
    if (S.L == 1024) tx_job_1024(P, G, S, jb, gsrc, wdst, scr, map, lane);
    else tx_job_512(P, G, S, jb, gsrc, wdst, scr, map, lane);
  }
}

__global__ void __launch_bounds__(FC_WARP_THREADS, 3)
k_rx_sync_warp(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, const FcChunk* __restrict__ chunks,
               int n_chunks, const float2* __restrict__ wave, float2* __restrict__ grid) {
  __shared__ FcPlanDev P;
  __shared__ int next_job;
  extern __shared__ __align__(16) float2 wscr[];
  load_plan_w(P, gP);
  const int stream = blockIdx.x / n_chunks;
  const FcChunk ch = chunks[blockIdx.x - stream * n_chunks];
  if (threadIdx.x == 0) next_job = ch.j0;
  __syncthreads();                                  // the plan copy is complete before any use
  const float2* src = wave + (size_t)stream * P.frame_len;
  float2* gdst = grid + (size_t)stream * P.grid_len;
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kScratch;
  float2* map = scr + kTrans;
  while (true) {
    int j = 0;
    if (lane == 0) j = atomicAdd(&next_job, 1);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= ch.j1) break;
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    const FcSubDev& S = P.s[G.first_sub];
    if (S.L == 1024) rx_job_1024(P, G, S, jb, src, gdst, scr, map, lane);
    else rx_job_512(P, G, S, jb, src, gdst, scr, map, lane);
  }
}

__global__ void k_zero(float4* __restrict__ p, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

size_t fc_warp_smem_bytes() { return (size_t)kWarps * kScratch * sizeof(float2); }

cudaError_t fc_launch_tx_sync_warp(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks,
                                   int n_streams, int frame_len, const float2* grid, float2* wave, cudaStream_t st) {
  int zero_in_kernel = n_chunks == 1;
  if (!zero_in_kernel) {
    const size_t n = (size_t)n_streams * frame_len;     // frame_len is even for this path
    k_zero<<<1024, 256, 0, st>>>(reinterpret_cast<float4*>(wave), n / 2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_tx_sync_warp<<<dim3((unsigned)(n_streams * n_chunks)), FC_WARP_THREADS, fc_warp_smem_bytes(), st>>>(
      dP, jobs, chunks, n_chunks, zero_in_kernel, grid, wave);
  return cudaGetLastError();
}

cudaError_t fc_launch_rx_sync_warp(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks,
                                   int n_streams, const float2* wave, float2* grid, cudaStream_t st) {
  k_rx_sync_warp<<<dim3((unsigned)(n_streams * n_chunks)), FC_WARP_THREADS, fc_warp_smem_bytes(), st>>>(
      dP, jobs, chunks, n_chunks, wave, grid);
  return cudaGetLastError();
}

cudaError_t fc_set_warp_smem_limits() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_tx_sync_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fc_warp_smem_bytes())))
    return e;
  return cudaFuncSetAttribute(k_rx_sync_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fc_warp_smem_bytes());
}

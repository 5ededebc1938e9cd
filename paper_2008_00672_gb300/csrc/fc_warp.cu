// Warp-centric symbol-synchronized FC kernels (sm_103a) for the numerologies
// with I = N/L = 2 and L in {512, 1024} (one subband per numerology group).
//
// One warp processes one symbol job (Sec. III-C for TX, Sec. IV for RX) end to
// end with no CTA-wide barrier:
//   * transforms are four-step FFTs held in registers (32 values per lane): one
//     1024-point transform (32 x 32) or two 512-point transforms (16 x 32), with
//     one shared-memory transpose each;
//   * the long N = 2048 transform is split by one radix-2 step into two
//     1024-point transforms (even and odd output samples for the TX IDFT, even
//     and odd bins for the RX DFT);
//   * the segmentation of the zero-padded symbol into the two FC blocks
//     (eq:padding, R_L^{(r)}) is a register renaming, because L/4 and L/2 are
//     multiples of the 32-sample stride of the register layout;
//   * TX overlap-add (blocks of a symbol, neighbouring symbols, numerology
//     groups; eq:multi-symb) is done with vector reductions into the zeroed
//     output waveform, so warps never wait for each other.
// A TX job is a short program of stages "prepare -> forward FFT -> consume" (inverse
// transforms as conj(FFT(conj(x)))), so the TX kernel holds a single copy of the
// unrolled FFT; RX jobs keep direction-specialised transforms in rolled loops (one copy
// of each per job shape). Each direction launches one kernel per job shape (the
// N = 2048 groups' jobs and the N = 1024 groups'), with the job inlined: a kernel then
// holds one shape's code, which the instruction cache keeps, and no calls (TX 1.395 ->
// 1.347 ms, RX 1.202 -> 1.066 ms at 2048 streams against one kernel for both shapes).
// Each launch takes the job-major list of its jobs over all streams, dealt to as many
// CTAs as the GPU holds at once.
#include <algorithm>

#include "fc_device.cuh"
#include "fc_internal.cuh"
#include "fc_warp_fft.cuh"

namespace {
using namespace fcdev;
using namespace fcwarp;

constexpr int kMap = 1024;                     // per-warp spectrum / re-layout buffer (float2)
constexpr int kScratch = kTrans + kMap;
constexpr int kWarps = FC_WARP_THREADS / 32;
// RX: one CTA of 12 warps per SM (the register file's limit at 168 registers), sharing the
// staged tables: per-lane step twiddles of 1024 points (32 rows) and 512 points (16 rows)
constexpr int kRxThreads = 384;
constexpr int kRxWarps = kRxThreads / 32;
constexpr int kRxTwiddles = 32 * 32 + 16 * 32;   // float2

// signed short-transform frequency of natural bin k (even L)
__device__ __forceinline__ int signed_bin(int k, int L) { return k < L / 2 ? k : k - L; }

// Twiddle tables of a job: 1024-point, and 512-point (L = 512) or 2048-point (N = 2048).
struct JobTables {
  const float2* t1024;
  const float2* t512;
  const float2* t2048;
};

// The TX kernel's tables staged in shared memory once per CTA: the per-lane step
// twiddles of the 512-point (16 rows) and 1024-point (32 rows) transforms, the full
// 2048-point forward table (the odd-sample rotation) and each group's TX weights (the bin
// loops read them at data-dependent positions; from shared memory they cost less than
// from the L1 cache).
constexpr int kTxTwiddles = 16 * 32 + 32 * 32 + 2048;   // float2
// The L = 512 kernel needs no 2048-point table; its warps hold a pair buffer (the second
// body of a pair of symbols) after their scratch instead.
constexpr int kPairBuf = 512;                              // float2
template <bool BIG> constexpr int kTxWarpScratch = BIG ? kScratch : kScratch + kPairBuf;
template <bool BIG> constexpr int kTxTables = BIG ? kTxTwiddles : kTxTwiddles - 2048;
struct TxTables {
  const float2* t1024;    // per-lane step table, 1024 points
  const float2* t512;     // per-lane step table, 512 points
  const float2* t2048;    // full forward table, 2048 points
};

__device__ __forceinline__ float weight_staged(const FcSubDev& S, const float* d, int p) {
  return (p >= S.p_lo && p < S.p_hi) ? d[p] : 0.f;
}

// ---------------------------------------------------------------------------
// TX job. L = 1024 (N = 2048), stages:
//   0   OFDM IDFT of the grid row -> body (kept in registers)
//   1/4 block r = 0/1: segment + window from the body, short DFT, map into the folded spectrum
//   2/5 even output samples of block r (IDFT of the folded spectrum), kept in registers
//   3/6 odd output samples (IDFT of the spectrum times exp(+j 2 pi q / 2048)); both
//       parities reduced into the waveform as float4
// L = 512 (N = 1024), a pair of symbols n, n + 1 (jb.nblk == 4) or a single symbol:
//   0   OFDM IDFT of both rows in one two-transform FFT (a single symbol: the second
//       transform's input is zero) -> body of n to the map buffer, body of n + 1 to the
//       warp's pair buffer
//   1   symbol s: both blocks segmented from its body, two 512-point DFTs (kept in registers)
//   2/3 symbol s, block r = 0/1: map into the 1024-bin spectrum, IDFT, reduce into the waveform
//   4-6 stages 1-3 for symbol n + 1 (pairs: the seven stages of an N = 2048 symbol)
// ---------------------------------------------------------------------------
// INIT (N = 2048 jobs of even n, one such group in the plan): the job writes its span
// [sigma_n, sigma_n + 3N/2) with stores instead of reductions (block 1 adds block 0's
// overlapping half, written by the same lane, before storing) and zeroes the samples up
// to the next even symbol (or the frame's end; the first one also those before it):
// this launch then initialises the whole waveform, which needs no memset, and the later
// launches reduce into it. Even symbols' spans are disjoint (2N + CPs > 3N/2 apart).
template <bool BIG, bool INIT, typename TI>
__device__ __forceinline__ void tx_job(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                       const TI* __restrict__ gsrc, float2* __restrict__ wdst, float2* scr,
                                       float2* map, float2* pbuf, int lane, const TxTables& tt, const float* wt,
                                       bool& waited) {
  constexpr bool big = BIG;                        // L = 1024 (N = 2048), else L = 512
  // pairs for complex64 input only: with BF16 loads the pair code grew the kernel past
  // what the instruction cache holds (1.49 -> 1.65 ms at 2048 streams)
  const bool pair = !big && std::is_same<TI, float2>::value && jb.nblk == 4;
  const JobTables tb{tt.t1024, tt.t512, tt.t2048};
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  const TI* __restrict__ row = gsrc + S.grid_off + (long long)jb.index * S.Lact;
  const bool ols = P.scheme_tx == FC_OLS;
  const int nN = big ? 2048 : 1024;
  const float2* __restrict__ twNg = P.sz[G.size_N].tw;                              // the plan's full table
  // the current symbol's CP lengths, position and phases (the second symbol of a pair
  // takes them over at stage 4)
  int lcp, ncp, start;
  float2 ph0, ph1;
  auto symbol = [&](int n) {
    lcp = S.lcp[n];
    ncp = G.ncp[n];
    start = G.offset + G.sigma[n];
    ph0 = root_pos(twNg, nN, (long long)S.c * G.cps[n]);                            // phi_0 theta_n
    ph1 = root_pos(twNg, nN, (long long)S.c * (G.cps[n] + G.N_S));                 // phi_1 theta_n
  };
  symbol(jb.index);
  const bool v4 = ((start & 1) == 0);
  const int nst = (big || pair) ? 7 : 4;
  float2 v[32], keep[32];
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    if (pair && st == 4) symbol(jb.index + 1);
    // ---------------- prepare ----------------
    bool inv, two512;
    if (big) {
      two512 = false;
      if (st == 0) {                                    // T1: active bins of the row
#pragma unroll
        for (int a = 0; a < 32; ++a) {
          const int f = signed_bin(32 * a + lane, 1024);
          v[a] = (f >= -hl && f < hu) ? ld_io(row + f + hl) : czero();
        }
        inv = true;
      } else if (st == 1 || st == 4) {                  // T2-T3: block r from the body
        const bool r1 = st == 4;
#pragma unroll
        for (int a = 0; a < 32; ++a) {
          const int t = 32 * a + lane;
          bool k;
          if (!ols) k = r1 ? (t >= 256 && t < 768) : (t >= 256 - lcp && t < 768);
          else k = r1 ? (t < 768) : (t >= 256 - lcp);
          const float2 b = r1 ? keep[(a + 8) & 31] : keep[(a + 24) & 31];
          v[a] = k ? b : czero();
        }
        inv = false;
      } else if (st == 2 || st == 5) {                  // T6: even samples from the folded spectrum;
#pragma unroll                                          //     the odd-sample input replaces it in place
        for (int a = 0; a < 32; ++a) {
          const int qp = 32 * a + lane;
          const float2 y = map[qp];
          int kt = (qp - S.c) & 1023;
          if (kt >= 512) kt -= 1024;
          v[a] = y;
          map[qp] = cmulc(y, tb.t2048[(S.c + kt) & 2047]);            // y exp(+j 2 pi q / 2048)
        }
        inv = true;
      } else {                                          // T6: odd samples; the even outputs move from
#pragma unroll                                          //     the transpose buffer into their map slots
        for (int a = 0; a < 32; ++a) {
          const int qp = 32 * a + lane;
          const float2 t = map[qp];
          map[qp] = scr[a * kPad + lane];
          v[a] = t;
        }
        inv = true;
      }
    } else {
      const int ss = (pair && st >= 4) ? st - 3 : st;   // stage of the current symbol
      if (st == 0) {
#pragma unroll
        for (int a = 0; a < 16; ++a) {
          const int f = signed_bin(32 * a + lane, 512);
          const bool in = f >= -hl && f < hu;
          v[a] = in ? ld_io(row + f + hl) : czero();
          v[16 + a] = (pair && in) ? ld_io(row + S.Lact + f + hl) : czero();
        }
        inv = true;
        two512 = true;
      } else if (ss == 1) {
        const float2* body = (st >= 4) ? pbuf : map;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
          for (int a = 0; a < 16; ++a) {
            const int t = 32 * a + lane;
            bool k;
            if (!ols) k = (r == 0) ? (t >= 128 - lcp && t < 384) : (t >= 128 && t < 384);
            else k = (r == 0) ? (t >= 128 - lcp) : (t < 384);
            v[16 * r + a] = k ? body[(t - 128 + 256 * r) & 511] : czero();
          }
        }
        __syncwarp();
        inv = false;
        two512 = true;
      } else {                                          // block r = ss - 2 into the 1024-bin spectrum
        const int r = ss - 2;
#pragma unroll
        for (int a = 0; a < 32; ++a) map[32 * a + lane] = czero();
        __syncwarp();
        if ((lane >> 4) == r) {
          const float2 ph = r ? ph1 : ph0;
#pragma unroll
          for (int k2 = 0; k2 < 32; ++k2) {
            const int kt = signed_bin((lane & 15) + 16 * k2, 512);
            map[(S.c + kt) & 1023] = cscale(cmul(keep[k2], ph), weight_staged(S, wt, kt + 256));
            if ((k2 & 7) == 7) sched_fence();
          }
        }
        __syncwarp();
#pragma unroll
        for (int a = 0; a < 32; ++a) v[a] = map[32 * a + lane];
        __syncwarp();
        inv = true;
        two512 = false;
      }
    }
    // ---------------- transform ----------------
    if (inv) conj32(v);
    warp_fft<true>(v, scr, tb.t1024, tb.t512, lane, two512);
    if (inv) conj32(v);
    // ---------------- consume ----------------
    if (big) {
      if (st == 0) {
#pragma unroll
        for (int k = 0; k < 32; ++k) keep[k] = v[k];   // body[k1 + 32 k2]
      } else if (st == 1 || st == 4) {                  // T5: shift, D_m, bin map with phi_r theta_n
        const float2 ph = (st == 4) ? ph1 : ph0;
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int kt = signed_bin(lane + 32 * k2, 1024);
          map[(S.c + kt) & 1023] = cscale(cmul(v[k2], ph), weight_staged(S, wt, kt + 512));
          if ((k2 & 7) == 7) sched_fence();
        }
        __syncwarp();
      } else if (st == 2 || st == 5) {                  // park the even outputs in this lane's
#pragma unroll                                          // column of the transpose buffer
        for (int k = 0; k < 32; ++k) scr[k * kPad + lane] = v[k];
      } else {                                          // T7: OLS window, R_N^{(r)}, Gamma_sigma
        const int r = (st == 6);
        const int lo = r ? G.N_L : G.N_L - ncp, hi = G.N_L + G.N_S;
        if (!waited) {                                  // the previous launch's waveform writes
          pdl_wait();
          waited = true;
        }
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int tau = 2 * (lane + 32 * k2);
          float2 a0 = map[32 * k2 + lane], a1 = v[k2];
          if (ols) {
            if (!(tau >= lo && tau < hi)) a0 = czero();
            if (!(tau + 1 >= lo && tau + 1 < hi)) a1 = czero();
          }
          float2* dst = wdst + start + r * 1024 + tau;
          if constexpr (INIT) {
            if (r && tau < 1024) {                      // block 0's second half, this lane's
              a0 = cadd(a0, dst[0]);
              a1 = cadd(a1, dst[1]);
            }
            if (v4) {
              *reinterpret_cast<float4*>(dst) = make_float4(a0.x, a0.y, a1.x, a1.y);
            } else {
              dst[0] = a0;
              dst[1] = a1;
            }
          } else if (v4) {
            atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a0.x, a0.y, a1.x, a1.y));
          } else {
            atomicAdd(dst, a0);
            atomicAdd(dst + 1, a1);
          }
        }
        __syncwarp();
      }
    } else {
      const int ss = (pair && st >= 4) ? st - 3 : st;
      if (st == 0) {                                    // body of n [k1 + 16 k2] from lanes 0..15 to
        if (lane < 16 || pair) {                        // the map buffer, body of n + 1 from lanes
          float2* body = (lane < 16) ? map : pbuf;      // 16..31 to the pair buffer
#pragma unroll
          for (int k2 = 0; k2 < 32; ++k2) body[(lane & 15) + 16 * k2] = v[k2];
        }
        __syncwarp();
      } else if (ss == 1) {
#pragma unroll
        for (int k = 0; k < 32; ++k) keep[k] = v[k];   // U_r[k1 + 16 k2], r = lane >> 4
      } else {
        const int r = ss - 2;
        const int lo = r ? G.N_L : G.N_L - ncp, hi = G.N_L + G.N_S;
        if (!waited) {
          pdl_wait();
          waited = true;
        }
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int tau = lane + 32 * k2;
          float2 a0 = v[k2];
          if (ols && !(tau >= lo && tau < hi)) a0 = czero();
          atomicAdd(wdst + start + r * 512 + tau, a0);
        }
      }
    }
  }
  if constexpr (INIT) {
    const int n = jb.index;
    const int end = n + 2 < G.B ? G.offset + G.sigma[n + 2] : P.frame_len;
    for (int t = start + 3 * G.N / 2 + lane; t < end; t += 32) wdst[t] = czero();
    if (n == 0)
      for (int t = lane; t < start; t += 32) wdst[t] = czero();
  }
}

// ---------------------------------------------------------------------------
// RX jobs: one function per numerology, each with its transforms specialised for
// their direction (they execute fewer instructions than conj(FFT(conj(x)))). The loops
// over blocks and bin parities stay rolled, so that each job holds one copy of each
// transform it uses (three for L = 1024 and three for L = 512): the instruction working
// set, more than the arithmetic, limits this kernel (rolling the L = 1024 job from seven
// inlined transforms to three took its time from 1.99 to 1.47 ms at 2048 streams, a few
// hundred bytes of spills included). The L = 1024 block loop carries only block 0's part
// of the symbol body into the block-1 iteration, which assembles and demodulates it.
// ---------------------------------------------------------------------------
template <int K, bool INV, bool STAGED = false>
__device__ __forceinline__ void step_twiddles_k(float2* v, const float2* __restrict__ tw, int lane) {
  if constexpr (STAGED) {             // per-lane step table in shared memory: row k holds W^(k lane)
#pragma unroll
    for (int k = 1; k < K; ++k) {
      float2 w = tw[k * 32 + lane];
      if (INV) w.y = -w.y;
      v[k] = cmul(v[k], w);
    }
    return;
  }
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
template <bool INV, bool STAGED = false>
__device__ __forceinline__ void warp_fft1024_d(float2 (&v)[32], float2* scr, const float2* __restrict__ tw, int lane) {
  Dft<32, INV>::run(v);
  step_twiddles_k<32, INV, STAGED>(v, tw, lane);
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
template <bool INV, bool STAGED = false>
__device__ __forceinline__ void warp_fft512x2_d(float2 (&v)[32], float2* scr, const float2* __restrict__ tw, int lane) {
  Dft<16, INV>::run(v);
  Dft<16, INV>::run(v + 16);
  {
    float2 t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t[k] = make_float2(1.f, 0.f);
    step_twiddles_k<16, INV, STAGED>(t, tw, lane);       // t[k] = W_512^{+-lane k}
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

// The RX kernel's tables staged in shared memory once per CTA: per-lane step twiddles of
// the 1024-point and 512-point transforms (rows of 32: row k holds W^(k lane)) and the
// job's group's RX weights.
struct RxStaged {
  const float2* s1024;
  const float2* s512;
  const float* w;
};

// ---------------------------------------------------------------------------
// RX, N = 2048, L = 1024
// ---------------------------------------------------------------------------
// j^e x for e mod 4 (multiplication by a power of +j)
__device__ __forceinline__ float2 mul_jpow(float2 x, int e) {
  switch (e & 3) {
    case 0: return x;
    case 1: return make_float2(-x.y, x.x);
    case 2: return make_float2(-x.x, -x.y);
    default: return make_float2(x.y, -x.x);
  }
}

// R1-R3 for block r: the 2048-point DFT as two 1024-point halves (even / odd bins),
// then the subband's 1024 bins gathered with conj(phi_r theta_n) and D_m into map
// at their natural short-transform index k. combine: instead of storing g_r[k],
// store j^k (g_r[k] - (-1)^k map[k]) (the bracket of eq:reduc, map holding g_1).
template <typename TI>
__device__ __forceinline__ void rx_block_gather_1024(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S,
                                                     const FcJob& jb, const TI* __restrict__ src, float2* scr,
                                                     float2* map, int lane, int r, bool combine, const RxStaged& st) {
  constexpr int L = 1024;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const TI* __restrict__ x = src + jb.start + r * (2048 / 2);
  const float2 ph = root_pos(twN, 2048, (long long)S.c * (G.cps[jb.index] + r * G.N_S));
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    float2 X[32];
    // even bins: DFT of x0 + x1; odd bins: DFT of (x0 - x1) exp(-j 2 pi tp / 2048)
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      const int tp = 32 * a + lane;
      const float2 x0 = ld_io(x + tp), x1 = ld_io(x + tp + 1024);
      X[a] = s ? cmul(csub(x0, x1), __ldg(twN + tp)) : cadd(x0, x1);
    }
    warp_fft1024_d<false, true>(X, scr, st.s1024, lane);     // bin 2 (k1 + 32 k2) + s
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int q = 2 * (lane + 32 * k2) + s;
      int kt = (q - S.c) & 2047;
      if (kt >= 1024) kt -= 2048;
      if (kt >= -L / 2 && kt < L / 2) {
        const int k = kt & (L - 1);
        const float2 g = cscale(cmulc(X[k2], ph), weight_staged(S, st.w, kt + L / 2));
        if (!combine) {
          map[k] = g;
        } else {
          const float2 g1 = map[k];
          map[k] = mul_jpow((k & 1) ? cadd(g, g1) : csub(g, g1), k);
        }
      }
    }
  }
}

// Overlap-save RX in the joint form of eq:reduc (opt-in, FC_FLAG_REDUCED_RX):
//   x_hat = W_L S_hat W_L^{-1} [j^k (g_0 - (-1)^k g_1)] + (-j)^k g_1   (scaled by L),
// where g_r are the gathered block spectra and S_hat keeps time samples [0, L/2).
// One IDFT and one DFT replace the two block IDFTs and the OFDM DFT (6 transforms of
// 1024 points per symbol instead of 7), at the cost of a second pass over the output row.
template <typename TI>
__device__ __forceinline__ void rx_job_1024_reduced(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                            const TI* __restrict__ src, float2* __restrict__ gdst, float2* scr,
                                            float2* map, int lane, const RxStaged& st) {
  constexpr int L = 1024;
  const int n = jb.index;
  const int hl = S.Lact / 2, hu = S.Lact - hl;
  float2* __restrict__ row = gdst + S.grid_off + (long long)n * S.Lact;
  float2 u[32];
  rx_block_gather_1024(P, G, S, jb, src, scr, map, lane, 1, false, st);    // map = g_1
  __syncwarp();
  // L (-j)^k g_1[k] goes straight to the output row; the same thread adds the
  // transform result to it at the end (no register copy across the next stages)
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const int k = lane + 32 * k2;
    const int f = k < L / 2 ? k : k - L;
    if (f >= -hl && f < hu) row[f + hl] = cscale(mul_jpow(map[k], 3 * k), (float)L);
  }
  __syncwarp();
  rx_block_gather_1024(P, G, S, jb, src, scr, map, lane, 0, true, st);     // map = j^k (g_0 - (-1)^k g_1)
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 32; ++a) u[a] = map[32 * a + lane];
  __syncwarp();
  warp_fft1024_d<true, true>(u, scr, st.s1024, lane);        // time k1 + 32 k2
#pragma unroll
  for (int k2 = 16; k2 < 32; ++k2) u[k2] = czero();   // S_hat
  warp_fft1024_d<false, true>(u, scr, st.s1024, lane);       // bin k1 + 32 k2
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const int bin = lane + 32 * k2;
    const int f = bin < L / 2 ? bin : bin - L;
    if (f >= -hl && f < hu) row[f + hl] = cadd(u[k2], row[f + hl]);
  }
}

// OLA: the scheme (a template parameter, so that the overlap-save form carries only the
// 16 values per lane it needs across the block loop)
template <bool OLA, typename TI, typename TO>
__device__ __forceinline__ void rx_job_1024(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                            const TI* __restrict__ src, TO* __restrict__ gdst, float2* scr,
                                            float2* map, int lane, const RxStaged& st) {
  constexpr int L = 1024;
  constexpr bool ola = OLA;
  constexpr int kCarry = OLA ? 24 : 16;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const int n = jb.index;
  // the part of the symbol body that block 0 contributes, x_ofdm[lane + 32 k] for k < 16
  // (OLS) or k < 24 (OLA), carried into the block-1 iteration, which assembles the body
  // and demodulates it
  float2 h0[kCarry];
#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
    // R1-R2: block r, radix-2 split of the 2048-point DFT into even (s = 0) and odd bins
    const TI* __restrict__ x = src + jb.start + r * (2048 / 2);
    float2 u[32];
    // R3: gather the subband's 1024 bins with conj(phi_r theta_n), D_m, inverse shift; the even
    // bins right after their transform, so only one half-spectrum is live in registers
    const float2 ph = root_pos(twN, 2048, (long long)S.c * (G.cps[n] + r * G.N_S));
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      if (s == 0) {
#pragma unroll
        for (int a = 0; a < 32; ++a) {
          const int tp = 32 * a + lane;
          float2 x0 = ld_io(x + tp), x1 = ld_io(x + tp + 1024);
          if (ola) {                               // A window [N_L, N_L + N_S) = [512, 1536)
            if (tp < 512) x0 = czero();
            if (tp >= 512) x1 = czero();
          }
          u[a] = cadd(x0, x1);
        }
      } else {
#pragma unroll
        for (int a = 0; a < 32; ++a) {
          const int tp = 32 * a + lane;
          float2 x0 = ld_io(x + tp), x1 = ld_io(x + tp + 1024);
          if (ola) {
            if (tp < 512) x0 = czero();
            if (tp >= 512) x1 = czero();
          }
          u[a] = cmul(csub(x0, x1), __ldg(twN + tp));   // (x0 - x1) exp(-j 2 pi tp / 2048)
        }
      }
      warp_fft1024_d<false, true>(u, scr, st.s1024, lane);     // bin 2 (k1 + 32 k2) + s
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int q = 2 * (lane + 32 * k2) + s;
        int kt = (q - S.c) & 2047;
        if (kt >= 1024) kt -= 2048;
        if (kt >= -L / 2 && kt < L / 2) {
          const float wt = weight_staged(S, st.w, kt + L / 2);
          map[kt & (L - 1)] = cscale(cmulc(u[k2], ph), wt);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 32; ++a) u[a] = map[32 * a + lane];
    __syncwarp();
    // R4: short IDFT
    warp_fft1024_d<true, true>(u, scr, st.s1024, lane);        // z_r[k1 + 32 k2] in u[k2]
    // R5: S window + concatenation (eq:concat2), or OLA of both blocks; x_ofdm[t], t = lane + 32 k
    if (r == 0) {
#pragma unroll
      for (int k = 0; k < kCarry; ++k) h0[k] = u[k + 8];
      continue;
    }
    float2 h[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (!OLA) h[k] = k < 16 ? h0[k] : u[k - 8];
      else h[k] = k < 8 ? h0[k] : (k < kCarry ? cadd(h0[k], u[k - 8]) : u[k - 8]);
    }
    // R6: OFDM demodulation and active-bin output
    warp_fft1024_d<false, true>(h, scr, st.s1024, lane);
    const int hl = S.Lact / 2, hu = S.Lact - hl;
    TO* __restrict__ row = gdst + S.grid_off + (long long)n * S.Lact;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int bin = lane + 32 * k2;
      const int f = bin < L / 2 ? bin : bin - L;
      if (f >= -hl && f < hu) st_io(row + f + hl, h[k2]);
    }
  }
}

// ---------------------------------------------------------------------------
// RX, N = 1024, L = 512
// ---------------------------------------------------------------------------
// A job is one symbol or a pair of symbols n, n + 1 (jb.nblk == 4): each symbol's two
// block DFTs, gather and short IDFTs, then the OFDM DFTs of both bodies as one
// two-transform FFT (a single symbol's second transform has a zero input). The first
// body waits in registers while the second symbol's blocks run.
template <typename TI, typename TO>
__device__ __forceinline__ void rx_job_512(const FcPlanDev& P, const FcGroupDev& G, const FcSubDev& S, const FcJob& jb,
                                           const TI* __restrict__ src, TO* __restrict__ gdst, float2* scr,
                                           float2* map, int lane, const RxStaged& st) {
  constexpr int L = 512;
  const float2* __restrict__ twN = P.sz[G.size_N].tw;
  const bool ola = P.scheme_rx == FC_OLA;
  const bool pair = jb.nblk == 4;
  float2 b0[16], v[32];
#pragma unroll 1
  for (int s = 0; s < (pair ? 2 : 1); ++s) {
    const int n = jb.index + s;
    const int start = G.offset + G.sigma[n];
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {                    // one copy of the block DFT in the code
      const TI* __restrict__ x = src + start + r * (1024 / 2);
      float2 u[32];
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        const int t = 32 * a + lane;
        float2 xv = ld_io(x + t);
        if (ola && !(t >= G.N_L && t < G.N_L + G.N_S)) xv = czero();
        u[a] = xv;
      }
      warp_fft1024_d<false, true>(u, scr, st.s1024, lane);     // bin k1 + 32 k2
      const float2 ph = root_pos(twN, 1024, (long long)S.c * (G.cps[n] + r * G.N_S));
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int q = lane + 32 * k2;
        int kt = (q - S.c) & 1023;
        if (kt >= 512) kt -= 1024;
        if (kt >= -L / 2 && kt < L / 2) {
          const float wt = weight_staged(S, st.w, kt + L / 2);
          map[r * L + (kt & (L - 1))] = cscale(cmulc(u[k2], ph), wt);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      v[a] = map[32 * a + lane];
      v[16 + a] = map[L + 32 * a + lane];
    }
    __syncwarp();
    warp_fft512x2_d<true, true>(v, scr, st.s512, lane);       // lane k1 + 16 r: z_r[k1 + 16 k2]
    {
      const int r = lane >> 4, k1 = lane & 15;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) map[r * L + k1 + 16 * k2] = v[k2];
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 16; ++a) {                   // the body of symbol n: x_T[32 a + lane]
      const int t = 32 * a + lane;
      float2 val;
      if (!ola) {
        val = t < L / 2 ? map[L / 4 + t] : map[L + t - L / 4];
      } else {
        val = czero();
        if (L / 4 + t < L) val = map[L / 4 + t];
        if (t >= L / 4) val = cadd(val, map[L + t - L / 4]);
      }
      if (s == 0) b0[a] = val;
      else v[16 + a] = val;
    }
    __syncwarp();
  }
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    v[a] = b0[a];
    if (!pair) v[16 + a] = czero();
  }
  warp_fft512x2_d<false, true>(v, scr, st.s512, lane);        // lane k1 + 16 T: X_T[k1 + 16 k2]
  const int sym = lane >> 4;
  if (sym == 0 || pair) {
    const int hl = S.Lact / 2, hu = S.Lact - hl;
    TO* __restrict__ row = gdst + S.grid_off + (long long)(jb.index + sym) * S.Lact;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int bin = (lane & 15) + 16 * k2;
      const int f = bin < L / 2 ? bin : bin - L;
      if (f >= -hl && f < hu) st_io(row + f + hl, v[k2]);
    }
  }
}


// ---------------------------------------------------------------------------
// kernels: the job-major item list of all streams (job j of every stream, one stream's
// jobs in cost order) dealt to the resident CTAs statically (CTA c takes items c, c + G,
// c + 2G, ...); a CTA's warps take its items through a shared counter. Every CTA gets the
// same mix of job shapes and the launch has no partial last wave.
// ---------------------------------------------------------------------------
// Ask L2 for [p, p + n): one 128-byte line per lane and step (p + n within the buffer).
template <typename T>
__device__ __forceinline__ void prefetch_l2(const T* p, int n, int lane) {
  constexpr int kLine = 128 / (int)sizeof(T);
  for (int i = kLine * lane; i < n; i += kLine * 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + i));
}

// RX job shapes: each runs in a kernel of its own, with its job function inlined (one
// shape's code per kernel, no calls). The eq:reduc form adds into its output row after
// storing to it, so it runs for complex64 output only; a BF16 output (rounded once per
// sample) takes the direct form.
enum RxShape { kRx1024Ols = 0, kRx1024Ola = 1, kRx512 = 2, kRx1024Reduced = 3 };

template <int SHAPE, typename TI, typename TO>
__device__ __forceinline__ void rx_run(const FcPlanDev& P, const FcJob& jb, const TI* __restrict__ src,
                                       TO* __restrict__ gdst, float2* scr, float2* map, int lane, const RxStaged& st) {
  const FcGroupDev& G = P.g[jb.group];
  const FcSubDev& S = P.s[G.first_sub];
  if constexpr (SHAPE == kRx1024Reduced) {
    if constexpr (std::is_same<TO, float2>::value) rx_job_1024_reduced(P, G, S, jb, src, gdst, scr, map, lane, st);
  } else if constexpr (SHAPE == kRx1024Ola) {
    rx_job_1024<true>(P, G, S, jb, src, gdst, scr, map, lane, st);
  } else if constexpr (SHAPE == kRx1024Ols) {
    rx_job_1024<false>(P, G, S, jb, src, gdst, scr, map, lane, st);
  } else {
    rx_job_512(P, G, S, jb, src, gdst, scr, map, lane, st);
  }
}

template <int SHAPE, typename TI, typename TO>
__global__ void __launch_bounds__(kRxThreads, 1)
k_rx_sync_warp(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, int n_jobs, int n_streams,
                     const TI* __restrict__ wave, TO* __restrict__ grid) {
  __shared__ FcPlanDev P;
  __shared__ int next_item;
  __shared__ int wt_off[FC_MAX_GROUPS];
  extern __shared__ __align__(16) float2 wscr[];
  pdl_trigger();
  load_plan_w(P, gP);
  if (threadIdx.x == 0) next_item = 0;
  __syncthreads();                                  // the plan copy is complete before any use
  // stage the per-lane step twiddles [1024: 32 rows | 512: 16 rows] and every group's weights
  float2* tabs = wscr + kRxWarps * kScratch;
  float* wts = reinterpret_cast<float*>(tabs + kRxTwiddles);
  for (int i = 0; i < P.n_sizes; ++i) {
    if (P.sz[i].n == 1024) stage_lane_twiddles(tabs, P.sz[i].tw, 1024, 32);
    if (P.sz[i].n == 512) stage_lane_twiddles(tabs + 1024, P.sz[i].tw, 512, 16);
  }
  {
    int off = 0;
    for (int g = 0; g < P.n_groups; ++g) {
      const FcSubDev& S = P.s[P.g[g].first_sub];
      if (threadIdx.x == 0) wt_off[g] = off;
      for (int p = threadIdx.x; p < S.L; p += blockDim.x) wts[off + p] = __ldg(S.drx + p);
      off += S.L;
    }
  }
  __syncthreads();
  const long long total = (long long)n_jobs * n_streams;
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kScratch;
  float2* map = scr + kTrans;
  while (true) {
    int u = 0;
    if (lane == 0) u = atomicAdd(&next_item, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    const long long item = blockIdx.x + (long long)u * gridDim.x;
    if (item >= total) break;
    const int j = (int)(item / n_streams);             // job-major: job j of every stream
    const int stream = (int)(item - (long long)j * n_streams);
    // the input of the CTA's next item (another stream, usually not in L2): both blocks
    // of the symbol, N + N/2 samples from its start, all of which that job reads
    const long long nx = item + gridDim.x;
    if (nx < total) {
      const int jn = (int)(nx / n_streams);
      const FcJob jbn = jobs[jn];
      const FcGroupDev& Gn = P.g[jbn.group];
      const int span = Gn.N + Gn.N / 2 + (jbn.nblk == 4 ? Gn.sigma[jbn.index + 1] - Gn.sigma[jbn.index] : 0);
      prefetch_l2(wave + (size_t)(nx - (long long)jn * n_streams) * P.frame_len + jbn.start, span, lane);
    }
    const FcJob jb = jobs[j];
    const RxStaged st{tabs, tabs + 1024, wts + wt_off[jb.group]};
    rx_run<SHAPE>(P, jb, wave + (size_t)stream * P.frame_len, grid + (size_t)stream * P.grid_len, scr, map, lane, st);
  }
  pdl_wait();               // a dependent launch completes after the launch before it
}

// TX: jobs of one stream run on several CTAs and reduce into the same waveform, which
// is zeroed beforehand. One kernel per job shape (BIG: the N = 2048 groups' jobs), so that
// each holds one shape's code.
template <bool BIG, bool INIT, typename TI>
__global__ void __launch_bounds__(FC_WARP_THREADS, FC_WARP_TX_MIN_BLOCKS)
k_tx_sync_warp(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, int n_jobs, int n_streams,
                     const TI* __restrict__ grid, float2* __restrict__ wave) {
  __shared__ FcPlanDev P;
  __shared__ int next_item;
  __shared__ int wt_off[FC_MAX_GROUPS];
  extern __shared__ __align__(16) float2 wscr[];
  pdl_trigger();
  load_plan_w(P, gP);
  if (threadIdx.x == 0) next_item = 0;
  __syncthreads();                                  // the plan copy is complete before any use
  // stage the tables: twiddles [512 | 1024 | 2048 (BIG only)], then every group's weights
  float2* tabs = wscr + kWarps * kTxWarpScratch<BIG>;
  float* wts = reinterpret_cast<float*>(tabs + kTxTables<BIG>);
  for (int i = 0; i < P.n_sizes; ++i) {
    const int n = P.sz[i].n;
    if (n == 512) stage_lane_twiddles(tabs, P.sz[i].tw, 512, 16);
    if (n == 1024) stage_lane_twiddles(tabs + 512, P.sz[i].tw, 1024, 32);
    if (BIG && n == 2048)                             // the odd-sample rotation of the N = 2048 jobs
      for (int m = threadIdx.x; m < n; m += blockDim.x) tabs[1536 + m] = __ldg(P.sz[i].tw + m);
  }
  {
    int off = 0;
    for (int g = 0; g < P.n_groups; ++g) {
      const FcSubDev& S = P.s[P.g[g].first_sub];
      if (threadIdx.x == 0) wt_off[g] = off;
      for (int p = threadIdx.x; p < S.L; p += blockDim.x) wts[off + p] = __ldg(S.dtx + p);
      off += S.L;
    }
  }
  __syncthreads();
  const TxTables tt{tabs + 512, tabs, BIG ? tabs + 1536 : nullptr};
  const long long total = (long long)n_jobs * n_streams;
  const int lane = threadIdx.x & 31;
  float2* scr = wscr + (threadIdx.x >> 5) * kTxWarpScratch<BIG>;
  float2* map = scr + kTrans;
  float2* pbuf = BIG ? nullptr : map + kMap;
  bool waited = false;
  while (true) {
    int u = 0;
    if (lane == 0) u = atomicAdd(&next_item, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    const long long item = blockIdx.x + (long long)u * gridDim.x;
    if (item >= total) break;
    const int j = (int)(item / n_streams);             // job-major: job j of every stream
    const int stream = (int)(item - (long long)j * n_streams);
    // the grid row of the CTA's next item (another stream, usually not in L2)
    const long long nx = item + gridDim.x;
    if (nx < total) {
      const int jn = (int)(nx / n_streams);
      const FcJob jbn = jobs[jn];
      const FcSubDev& Sn = P.s[P.g[jbn.group].first_sub];
      prefetch_l2(grid + (size_t)(nx - (long long)jn * n_streams) * P.grid_len + Sn.grid_off +
                      (long long)jbn.index * Sn.Lact,
                  (jbn.nblk == 4 ? 2 : 1) * Sn.Lact, lane);
    }
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    tx_job<BIG, INIT>(P, G, P.s[G.first_sub], jb, grid + (size_t)stream * P.grid_len, wave + (size_t)stream * P.frame_len, scr,
           map, pbuf, lane, tt, wts + wt_off[jb.group], waited);
  }
}


}  // namespace

// the TX kernels' dynamic shared memory: per-warp scratch + staged twiddles + weights
static size_t tx_smem_bytes(bool big, int weight_floats) {
  const int scratch = big ? kTxWarpScratch<true> : kTxWarpScratch<false>;
  const int twiddles = big ? kTxTables<true> : kTxTables<false>;
  return ((size_t)kWarps * scratch + twiddles) * sizeof(float2) + (((size_t)weight_floats * 4 + 15) & ~(size_t)15);
}

template <bool BIG, bool INIT, typename TI>
static cudaError_t launch_tx_warp(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_streams, size_t smem,
                                  const TI* grid, float2* wave, int num_sms, cudaStream_t st, bool& pdl) {
  if (n_jobs < 1) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tx_sync_warp<BIG, INIT, TI>, FC_WARP_THREADS, smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n_jobs * n_streams;
  long long ctas = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
  if (ctas > total) ctas = total;
  if (ctas < 1) return cudaSuccess;
  e = fcwarp::launch_k(k_tx_sync_warp<BIG, INIT, TI>, (unsigned)ctas, FC_WARP_THREADS, smem, st, pdl, dP, jobs,
                       n_jobs, n_streams, grid, wave);
  pdl = true;                                        // the call's next launch may overlap this one's tail
  return e;
}

template <typename TI>
static cudaError_t launch_tx_shapes(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_init, int n_big,
                                    int n_streams, int weight_floats, const TI* grid, float2* wave, int num_sms,
                                    cudaStream_t st) {
  const size_t big = tx_smem_bytes(true, weight_floats);
  bool pdl = false;                                  // the first launch follows the stream's earlier work
  cudaError_t e = launch_tx_warp<true, true>(dP, jobs, n_init, n_streams, big, grid, wave, num_sms, st, pdl);
  if (e != cudaSuccess) return e;
  e = launch_tx_warp<true, false>(dP, jobs + n_init, n_big - n_init, n_streams, big, grid, wave, num_sms, st, pdl);
  if (e != cudaSuccess) return e;
  return launch_tx_warp<false, false>(dP, jobs + n_big, n_jobs - n_big, n_streams, tx_smem_bytes(false, weight_floats),
                                      grid, wave, num_sms, st, pdl);
}

cudaError_t fc_launch_tx_sync_warp(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_init, int n_big,
                                   int n_streams, int frame_len, int weight_floats, const void* grid, int grid_bf16,
                                   float2* wave, int num_sms, cudaStream_t st) {
  if (n_init == 0) {                                // no initialising launch: zero the waveform
    cudaError_t e = cudaMemsetAsync(wave, 0, (size_t)n_streams * frame_len * sizeof(float2), st);
    if (e != cudaSuccess) return e;
  }
  return grid_bf16 ? launch_tx_shapes(dP, jobs, n_jobs, n_init, n_big, n_streams, weight_floats, (const bf2*)grid,
                                      wave, num_sms, st)
                   : launch_tx_shapes(dP, jobs, n_jobs, n_init, n_big, n_streams, weight_floats, (const float2*)grid,
                                      wave, num_sms, st);
}

static size_t rx_smem_bytes(int weight_floats) {
  return (size_t)kRxWarps * kScratch * sizeof(float2) + (size_t)kRxTwiddles * sizeof(float2) +
         (((size_t)weight_floats * 4 + 15) & ~(size_t)15);
}

template <int SHAPE, typename TI, typename TO>
static cudaError_t launch_rx_warp(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_streams, size_t smem,
                                  const void* wave, void* grid, int num_sms, cudaStream_t st, bool& pdl) {
  if (n_jobs < 1) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rx_sync_warp<SHAPE, TI, TO>, kRxThreads, smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n_jobs * n_streams;
  long long ctas = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
  if (ctas > total) ctas = total;
  if (ctas < 1) return cudaSuccess;
  e = fcwarp::launch_k(k_rx_sync_warp<SHAPE, TI, TO>, (unsigned)ctas, kRxThreads, smem, st, pdl, dP, jobs, n_jobs,
                       n_streams, (const TI*)wave, (TO*)grid);
  pdl = true;
  return e;
}

template <typename TO>
static cudaError_t launch_rx_shapes(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_big, int n_streams,
                                    size_t smem, const void* wave, void* grid, int big_shape, int num_sms,
                                    cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  bool pdl = false;                                  // the first launch follows the stream's earlier work
  // the N = 1024 jobs first: measured 1 % faster than the other order (the N = 2048
  // kernel's longer jobs then start under the first kernel's tail)
  e = launch_rx_warp<kRx512, float2, TO>(dP, jobs + n_big, n_jobs - n_big, n_streams, smem, wave, grid, num_sms, st,
                                         pdl);
  if (e != cudaSuccess) return e;
  if (big_shape == kRx1024Ola) {
    e = launch_rx_warp<kRx1024Ola, float2, TO>(dP, jobs, n_big, n_streams, smem, wave, grid, num_sms, st, pdl);
  } else {
    bool done = false;
    if constexpr (std::is_same<TO, float2>::value) {
      if (big_shape == kRx1024Reduced) {
        e = launch_rx_warp<kRx1024Reduced, float2, TO>(dP, jobs, n_big, n_streams, smem, wave, grid, num_sms, st,
                                                       pdl);
        done = true;
      }
    }
    if (!done)
      e = launch_rx_warp<kRx1024Ols, float2, TO>(dP, jobs, n_big, n_streams, smem, wave, grid, num_sms, st, pdl);
  }
  return e;
}

cudaError_t fc_launch_rx_sync_warp(const FcPlanDev* dP, const FcJob* jobs, int n_jobs, int n_big, int n_streams,
                                   int weight_floats, int scheme_rx, int flags, const void* wave, void* grid, int io,
                                   int num_sms, cudaStream_t st) {
  const size_t smem = rx_smem_bytes(weight_floats);
  const int big_shape = scheme_rx == FC_OLA ? kRx1024Ola
                        : ((flags & FC_FLAG_REDUCED_RX) && !(io & FC_IO_OUT_BF16)) ? kRx1024Reduced
                                                                                   : kRx1024Ols;
  // complex64 input (a BF16 waveform is widened beforehand: the BF16 loads would grow
  // the L = 1024 job past what the instruction cache holds, which doubled its time)
  switch (io & (FC_IO_IN_BF16 | FC_IO_OUT_BF16)) {
    case 0:
      return launch_rx_shapes<float2>(dP, jobs, n_jobs, n_big, n_streams, smem, wave, grid, big_shape, num_sms, st);
    case FC_IO_OUT_BF16:
      return launch_rx_shapes<bf2>(dP, jobs, n_jobs, n_big, n_streams, smem, wave, grid, big_shape, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
// Sample-type conversion of a buffer: complex64 rounded once to complex BF16 (the warp TX
// kernel's accumulated waveform into a BF16 output), or complex BF16 widened exactly to
// complex64 (a BF16 waveform into the warp RX kernel).
template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ src, TO* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    st_io(dst + i, ld_io(src + i));
}

template <typename TI, typename TO>
cudaError_t launch_convert(const TI* src, TO* dst, long long n, int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long ctas = (n + 255) / 256;
  if (ctas > 8LL * num_sms) ctas = 8LL * num_sms;
  k_convert<<<dim3((unsigned)ctas), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
}  // namespace

cudaError_t fc_launch_to_bf16(const float2* src, void* dst, long long n, int num_sms, cudaStream_t st) {
  return launch_convert(src, (bf2*)dst, n, num_sms, st);
}

cudaError_t fc_launch_from_bf16(const void* src, float2* dst, long long n, int num_sms, cudaStream_t st) {
  return launch_convert((const bf2*)src, dst, n, num_sms, st);
}

cudaError_t fc_set_warp_smem_limits() {
  cudaError_t e;
  const int tx = (int)std::max(tx_smem_bytes(true, FC_MAX_GROUPS * 1024), tx_smem_bytes(false, FC_MAX_GROUPS * 1024));
  const int rx = (int)rx_smem_bytes(FC_MAX_GROUPS * 1024);
  const void* tx_kernels[] = {
      (const void*)k_tx_sync_warp<true, true, float2>, (const void*)k_tx_sync_warp<true, false, float2>,
      (const void*)k_tx_sync_warp<false, false, float2>, (const void*)k_tx_sync_warp<true, true, bf2>,
      (const void*)k_tx_sync_warp<true, false, bf2>, (const void*)k_tx_sync_warp<false, false, bf2>};
  for (const void* k : tx_kernels)
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tx))) return e;
  const void* rx_kernels[] = {
      (const void*)k_rx_sync_warp<kRx1024Ols, float2, float2>, (const void*)k_rx_sync_warp<kRx1024Ola, float2, float2>,
      (const void*)k_rx_sync_warp<kRx512, float2, float2>, (const void*)k_rx_sync_warp<kRx1024Reduced, float2, float2>,
      (const void*)k_rx_sync_warp<kRx1024Ols, float2, bf2>, (const void*)k_rx_sync_warp<kRx1024Ola, float2, bf2>,
      (const void*)k_rx_sync_warp<kRx512, float2, bf2>};
  for (const void* k : rx_kernels)
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, rx))) return e;
  return cudaSuccess;
}

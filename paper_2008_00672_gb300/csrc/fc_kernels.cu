// CUDA kernels (sm_103a) of FC-filtered CP-OFDM TX synthesis and RX analysis.
//
// Structure (plain FP32 path):
//   * every transform (OFDM IDFT/DFT L_OFDM, short DFT/IDFT L_m, long IDFT/DFT N)
//     is an in-place mixed-radix Stockham FFT in shared memory, one CTA per job,
//     radix-2/3/4/8/16 butterflies in registers, FP32 twiddles generated in FP64
//     on the host and rounded once;
//   * the spectra of a block never leave shared memory: the short-DFT output is
//     weighted by D_m and scattered through the bin map Xi straight into the
//     long spectrum (TX), or gathered from it (RX);
//   * TX output assembly (OLA accumulate, OLS discard, symbol-wise OLA with the
//     Gamma_sigma placement of eq:multi-symb, and the sum over subbands and
//     numerology groups) happens in a shared-memory ring that each CTA owns for
//     a contiguous range of output time; a range is written to HBM exactly once,
//     when no later job can touch it;
//   * every transform buffer in shared memory holds logical element l at index
//     l + l/16 (one float2 of padding after every 16, see sp()).
//
// Symbol-synchronized jobs are (group, symbol) pairs and process the two FC
// blocks of a symbol as a batch of two (Sec. III-C); continuous jobs are pairs
// of consecutive FC blocks (Sec. III-B).
#include <cuda_bf16.h>

#include "fc_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// I/O samples: complex64 (float2) or complex BF16 (bf2 = {re, im}); the arithmetic is
// FP32 either way, and a BF16 output is rounded once, to nearest, ties to even.
using bf2 = __nv_bfloat162;
__device__ __forceinline__ float2 io_ld(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 io_ld(const bf2* p) { return __bfloat1622float2(__ldg(p)); }
__device__ __forceinline__ void io_st(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void io_st(bf2* p, float2 v) { *p = __float22bfloat162_rn(v); }

// Physical index of logical element l of a transform buffer in shared memory. One float2
// of padding after every 16 spreads the first Stockham pass's stores (R consecutive
// outputs per thread, a stride of R float2 across the warp) over distinct banks, and
// keeps the unit-stride accesses of the other passes conflict-free. A buffer of logical
// length n takes fc_padded_len(n) elements.
__device__ __forceinline__ int sp(int l) { return l + (l >> 4); }

// multiply by -i (forward transform) or +i (inverse transform)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi m / 16), m in [0, 16)
__host__ __device__ constexpr float c16(int m) {
  return m == 0 ? 1.0f
       : m == 1 ? 0.92387953251128674f
       : m == 2 ? 0.70710678118654752f
       : m == 3 ? 0.38268343236508977f
       : m == 4 ? 0.0f
       : m == 5 ? -0.38268343236508977f
       : m == 6 ? -0.70710678118654752f
       : m == 7 ? -0.92387953251128674f
       : m == 8 ? -1.0f
       : m == 9 ? -0.92387953251128674f
       : m == 10 ? -0.70710678118654752f
       : m == 11 ? -0.38268343236508977f
       : m == 12 ? 0.0f
       : m == 13 ? 0.38268343236508977f
       : m == 14 ? 0.70710678118654752f
                 : 0.92387953251128674f;
}

// a * exp(-+ j 2 pi M / 16): minus sign for the forward DFT, plus for the inverse
template <int M, bool INV>
__device__ __forceinline__ float2 tw16(float2 a) {
  constexpr int m = M & 15;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 4) {
    return mul_mi<INV>(a);
  } else if constexpr (m == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (m == 12) {
    return mul_mi<!INV>(a);
  } else {
    constexpr float c = c16(m);
    constexpr float s = c16((m + 12) & 15);   // sin(2 pi m/16)
    if constexpr (INV) return make_float2(a.x * c - a.y * s, a.y * c + a.x * s);
    else return make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
  }
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// In-register DFT of size R (X[k] = sum_t x[t] exp(-+ j 2 pi k t / R)), natural order.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2 (&v)[2]) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <bool INV>
struct Dft<3, INV> {
  static __device__ __forceinline__ void run(float2 (&v)[3]) {
    const float s = 0.86602540378443865f;   // sin(2 pi/3); cos(2 pi/3) = -1/2
    const float2 s12 = cadd(v[1], v[2]), d12 = csub(v[1], v[2]);
    const float2 m = make_float2(fmaf(-0.5f, s12.x, v[0].x), fmaf(-0.5f, s12.y, v[0].y));
    const float2 isd = make_float2(-s * d12.y, s * d12.x);   // j s (x1 - x2)
    v[0] = cadd(v[0], s12);
    if (INV) {
      v[1] = cadd(m, isd);
      v[2] = csub(m, isd);
    } else {
      v[1] = csub(m, isd);
      v[2] = cadd(m, isd);
    }
  }
};

template <bool INV>
struct Dft<4, INV> {
  static __device__ __forceinline__ void run(float2 (&v)[4]) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};

// 8 = 2 x 4: inner 2-point DFTs over t1 (stride 4), twiddle W_8^{t2 k1}, outer 4-point DFTs.
template <bool INV>
struct Dft<8, INV> {
  static __device__ __forceinline__ void run(float2 (&v)[8]) {
#pragma unroll
    for (int t2 = 0; t2 < 4; ++t2) {
      const float2 a = v[t2];
      v[t2] = cadd(a, v[t2 + 4]);
      v[t2 + 4] = csub(a, v[t2 + 4]);
    }
    v[5] = tw16<2, INV>(v[5]);
    v[6] = tw16<4, INV>(v[6]);
    v[7] = tw16<6, INV>(v[7]);
    dft4<INV>(v[0], v[1], v[2], v[3]);
    dft4<INV>(v[4], v[5], v[6], v[7]);
    // v[4 k1 + k2] holds X[k1 + 2 k2]
    float2 t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 2 * k2] = t[4 * k1 + k2];
  }
};

// 16 = 4 x 4: inner 4-point DFTs over t1 (stride 4), twiddle W_16^{t2 k1}, outer 4-point DFTs.
template <bool INV>
struct Dft<16, INV> {
  static __device__ __forceinline__ void run(float2 (&v)[16]) {
#pragma unroll
    for (int t2 = 0; t2 < 4; ++t2) dft4<INV>(v[t2], v[t2 + 4], v[t2 + 8], v[t2 + 12]);
    v[5] = tw16<1, INV>(v[5]);
    v[6] = tw16<2, INV>(v[6]);
    v[7] = tw16<3, INV>(v[7]);
    v[9] = tw16<2, INV>(v[9]);
    v[10] = tw16<4, INV>(v[10]);
    v[11] = tw16<6, INV>(v[11]);
    v[13] = tw16<3, INV>(v[13]);
    v[14] = tw16<6, INV>(v[14]);
    v[15] = tw16<9, INV>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
  }
};

// One register file v[] serves every radix: butterfly u of a thread occupies
// v[u R .. u R + R). The radix-specific phases contain no barrier, so the
// register allocator sees a single live array across the pass.
// Butterfly idx of a pass -> (transform b, butterfly i within it, k = i mod p), without
// a division where it can: batch is 1 or 2, and p is a power of two until the radix-3
// passes (pm = p - 1 then, else -1).
__device__ __forceinline__ void butterfly_of(int idx, int nb, int p, int pm, int& b, int& i, int& k) {
  b = 0;
  i = idx;
  while (i >= nb) {
    i -= nb;
    ++b;
  }
  k = pm >= 0 ? (i & pm) : i % p;
}

template <int R, bool INV>
__device__ __forceinline__ void pass_load(float2 (&v)[FC_MAX_ELEMS_PER_THREAD], const float2* a, int n, int batch,
                                          int p, const float2* __restrict__ tw) {
  constexpr int MAXB = FC_MAX_ELEMS_PER_THREAD / R;
  const int nb = n / R;
  const int total = nb * batch;
  const int twstep = n / (p * R);
  const int pm = (p & (p - 1)) == 0 ? p - 1 : -1;
#pragma unroll
  for (int u = 0; u < MAXB; ++u) {
    const int idx = threadIdx.x + u * FC_THREADS;
    if (idx < total) {
      int b, i, k;
      butterfly_of(idx, nb, p, pm, b, i, k);
      const int s = b * n + i;
      float2 w[R];
#pragma unroll
      for (int j = 0; j < R; ++j) w[j] = a[sp(s + j * nb)];
      if (p > 1) {
        // W_{pR}^{j k} is read from the table for j a power of two and formed as the
        // product W^{(j - h) k} W^{h k} (h the highest power of two in j) otherwise:
        // 4 table reads instead of 15 for radix 16, at most three roundings more.
        float2 t[R];
#pragma unroll
        for (int j = 1; j < R; ++j) {
          if ((j & (j - 1)) == 0) {
            t[j] = __ldg(tw + j * k * twstep);
            if (INV) t[j].y = -t[j].y;
          } else {
            int h = 1;
            while (2 * h <= j) h *= 2;
            t[j] = cmul(t[j - h], t[h]);
          }
        }
#pragma unroll
        for (int j = 1; j < R; ++j) w[j] = cmul(w[j], t[j]);
      }
      Dft<R, INV>::run(w);
#pragma unroll
      for (int j = 0; j < R; ++j) v[u * R + j] = w[j];
    }
  }
}

template <int R>
__device__ __forceinline__ void pass_store(const float2 (&v)[FC_MAX_ELEMS_PER_THREAD], float2* a, int n, int batch,
                                           int p) {
  constexpr int MAXB = FC_MAX_ELEMS_PER_THREAD / R;
  const int nb = n / R;
  const int total = nb * batch;
  const int pm = (p & (p - 1)) == 0 ? p - 1 : -1;
#pragma unroll
  for (int u = 0; u < MAXB; ++u) {
    const int idx = threadIdx.x + u * FC_THREADS;
    if (idx < total) {
      int b, i, k;
      butterfly_of(idx, nb, p, pm, b, i, k);
      const int d = b * n + (i - k) * R + k;
#pragma unroll
      for (int j = 0; j < R; ++j) a[sp(d + j * p)] = v[u * R + j];
    }
  }
}

// In-place Stockham FFT over `batch` (1 or 2) contiguous transforms of size n in a
// padded shared-memory buffer (logical index l at sp(l)). Pass s with radix R and p =
// product of the previous radices:
//   butterfly i (0 <= i < n/R), k = i mod p, inputs a[i + j n/R] * W_{pR}^{j k},
//   DFT_R, outputs to a[(i - k) R + k + j p]. All threads read their butterflies
//   into registers, synchronise, then write back, so one buffer suffices.
//   Requires batch * n <= FC_THREADS * FC_MAX_ELEMS_PER_THREAD (radix 3:
//   batch * n / 3 <= FC_THREADS * floor(FC_MAX_ELEMS_PER_THREAD / 3)).
// Unnormalised DFT (INV=false, exp(-j...)) or inverse DFT without 1/n (INV=true).
template <bool INV>
__device__ __forceinline__ void fft_inplace(float2* a, int batch, const FcSize& z) {
  float2 v[FC_MAX_ELEMS_PER_THREAD];
  int p = 1;
#pragma unroll 1
  for (int s = 0; s < z.npass; ++s) {
    const int R = z.radix[s];
    if (R == 16) pass_load<16, INV>(v, a, z.n, batch, p, z.tw);
    else if (R == 8) pass_load<8, INV>(v, a, z.n, batch, p, z.tw);
    else if (R == 4) pass_load<4, INV>(v, a, z.n, batch, p, z.tw);
    else if (R == 2) pass_load<2, INV>(v, a, z.n, batch, p, z.tw);
    else pass_load<3, INV>(v, a, z.n, batch, p, z.tw);
    __syncthreads();
    if (R == 16) pass_store<16>(v, a, z.n, batch, p);
    else if (R == 8) pass_store<8>(v, a, z.n, batch, p);
    else if (R == 4) pass_store<4>(v, a, z.n, batch, p);
    else if (R == 2) pass_store<2>(v, a, z.n, batch, p);
    else pass_store<3>(v, a, z.n, batch, p);
    __syncthreads();
    p *= R;
  }
}

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_plan(FcPlanDev& P, const FcPlanDev* __restrict__ gP) {
  const int words = (int)(sizeof(FcPlanDev) / 4);
  const int* src = reinterpret_cast<const int*>(gP);
  int* dst = reinterpret_cast<int*>(&P);
  for (int i = threadIdx.x; i < words; i += FC_THREADS) dst[i] = __ldg(src + i);
  __syncthreads();
}

__device__ __forceinline__ void zero_buf(float2* a, int n) {
  for (int i = threadIdx.x; i < n; i += FC_THREADS) a[i] = make_float2(0.f, 0.f);
}

// exp(+j 2 pi e / N) from the forward twiddle table of size N, e reduced exactly.
__device__ __forceinline__ float2 pos_root(const FcSize& z, long long e) {
  long long m = e % z.n;
  if (m < 0) m += z.n;
  float2 w = __ldg(z.tw + m);
  return make_float2(w.x, -w.y);
}

// bin i of an n-point DFT -> index of the active subcarrier (or -1)
__device__ __forceinline__ int active_index(int i, int n, int n_act) {
  const int f = (i < (n + 1) / 2) ? i : i - n;
  const int lo = n_act / 2;
  return (f >= -lo && f < n_act - lo) ? f + lo : -1;
}

// The TX ring holds output time T at ring[T mod RS]; RS (the longest job span rounded
// up, at least FC_THREADS) need not be a power of two, so a thread steps its index by
// FC_THREADS and wraps it.
__device__ __forceinline__ int ring_step(int r, int RS) {
  r += FC_THREADS;
  return r >= RS ? r - RS : r;
}

// Copy ring[from, to) to dst and clear it, in segments no longer than the ring.
template <typename TO>
__device__ __forceinline__ void ring_flush(float2* ring, int RS, TO* __restrict__ dst, int from, int to) {
  while (from < to) {
    const int seg = min(to - from, RS);
    int r = ((from + (int)threadIdx.x) % RS + RS) % RS;
    for (int i = threadIdx.x; i < seg; i += FC_THREADS, r = ring_step(r, RS)) {
      io_st(dst + from + i, ring[r]);
      ring[r] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    from += seg;
  }
}

// OFDM modulation of one symbol into buf[0, Lofdm): active bins, inverse DFT (unscaled).
template <typename TI>
__device__ __forceinline__ void ofdm_symbol_to_time(const FcPlanDev& P, const FcSubDev& S, const TI* __restrict__ row,
                                                    float2* buf) {
  const int L = S.Lofdm;
  for (int i = threadIdx.x; i < L; i += FC_THREADS) {
    const int a = active_index(i, L, S.Lact);
    buf[sp(i)] = a >= 0 ? io_ld(row + a) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_inplace<true>(buf, 1, P.sz[S.size_O]);
}

// TX map: Y[r][(c + p - floor(L/2)) mod N] += Z[r][(p - floor(L/2)) mod L] * D[p] * ph_r
__device__ __forceinline__ void tx_map(const FcSubDev& S, int N, const float2* Z, float2* Y, float2 ph0, float2 ph1,
                                       int nblk) {
  const int L = S.L, h = L / 2, cnt = S.p_hi - S.p_lo;
  for (int idx = threadIdx.x; idx < nblk * cnt; idx += FC_THREADS) {
    const int r = idx >= cnt;
    const int p = S.p_lo + idx - r * cnt;
    int k = p - h;
    if (k < 0) k += L;
    int q = S.c + p - h;                               // c in [0, N), |p - h| <= L/2 <= N/2
    q += q < 0 ? N : (q >= N ? -N : 0);
    const float w = __ldg(S.dtx + p);
    const float2 v = cmul(Z[sp(r * L + k)], r ? ph1 : ph0);
    float2& y = Y[sp(r * N + q)];
    y.x = fmaf(v.x, w, y.x);
    y.y = fmaf(v.y, w, y.y);
  }
  __syncthreads();
}

// RX gather: V[r][k] = Y[r][(c + p - floor(L/2)) mod N] * conj(ph_r) * Drx[p], p = (k + floor(L/2)) mod L
__device__ __forceinline__ void rx_gather(const FcSubDev& S, int N, const float2* Y, float2* V, float2 ph0, float2 ph1,
                                          int nblk) {
  const int L = S.L, h = L / 2;
  for (int idx = threadIdx.x; idx < 2 * L; idx += FC_THREADS) {
    const int r = idx >= L;
    const int k = idx - r * L;
    int p = k + h;
    if (p >= L) p -= L;
    float2 v = make_float2(0.f, 0.f);
    if (r < nblk && p >= S.p_lo && p < S.p_hi) {
      int q = S.c + p - h;
      q += q < 0 ? N : (q >= N ? -N : 0);
      const float2 ph = r ? ph1 : ph0;
      const float2 y = Y[sp(r * N + q)];
      const float w = __ldg(S.drx + p);
      // y * conj(ph) * w
      v = make_float2((y.x * ph.x + y.y * ph.y) * w, (y.y * ph.x - y.x * ph.y) * w);
    }
    V[sp(idx)] = v;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Symbol-synchronized TX (Sec. III-C..E)
// ---------------------------------------------------------------------------
// One chunk of one stream: the CTA runs the chunk's symbol jobs in order and owns
// the output samples [ch.t0, ch.t1) of the stream (written once, from the ring).
template <typename TI, typename TO>
__device__ __forceinline__ void tx_sync_chunk(const FcPlanDev& P, const FcJob* __restrict__ jobs, const FcChunk ch,
                                              int stream, const TI* __restrict__ grid, TO* __restrict__ wave,
                                              unsigned char* smem_raw) {
  float2* ring = reinterpret_cast<float2*>(smem_raw);
  float2* Y = ring + P.ring;
  float2* W = Y + P.ybuf;
  const int RS = P.ring;
  const bool io_time = (P.flags & FC_FLAG_IO_TIME) != 0;
  const TI* gsrc = grid + (size_t)stream * (io_time ? P.time_tx_len : P.grid_len);
  TO* wdst = wave + (size_t)stream * P.frame_len;
  zero_buf(ring, RS);
  int flushed = ch.t0;
  __syncthreads();

  for (int j = ch.j0; j < ch.j1; ++j) {
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    const int N = G.N, n = jb.index;
    zero_buf(Y, fc_padded_len(2 * N));
    __syncthreads();
    for (int m = G.first_sub; m < G.first_sub + G.n_sub; ++m) {
      const FcSubDev& S = P.s[m];
      const int L = S.L, q4 = L / 4;
      const int lcp = S.lcp[n];
      // T1: OFDM symbol (eq:TX_OFDMmod, scaling folded into D); time-domain input: the
      // caller's CP and body, brought to the same scale (sqrt(L_OFDM))
      const TI* tin = gsrc + S.time_tx_off + S.soff[n];
      if (!io_time) ofdm_symbol_to_time(P, S, gsrc + S.grid_off + (long long)n * S.Lact, W);
      // T2-T3: CP insertion, zero padding to 3L/2 (eq:padding), two segments with the
      // dynamic-overlap analysis windows a_{m,0}, a_{m,1} (OLA) or none (OLS)
      float2* Z = W + fc_padded_len(L);
      for (int idx = threadIdx.x; idx < 2 * L; idx += FC_THREADS) {
        const int r = idx >= L;
        const int zi = r * (L / 2) + idx - r * L;     // index in the padded symbol z_n
        bool in = zi >= q4 - lcp && zi < q4 + L;
        if (P.scheme_tx == FC_OLA) in = in && (r == 0 ? zi < 3 * q4 : zi >= 3 * q4);
        float2 v = make_float2(0.f, 0.f);
        if (in && io_time) {
          v = cscale(io_ld(tin + zi - (q4 - lcp)), sqrtf((float)S.Lofdm));
        } else if (in) {
          int bi = zi - q4;
          if (bi < 0) bi += L;
          v = W[sp(bi)];
        }
        Z[sp(idx)] = v;
      }
      __syncthreads();
      // T4: short DFTs of both blocks
      fft_inplace<false>(Z, 2, P.sz[S.size_L]);
      // T5: fftshift, D_m, bin map with phi_r theta_n (phi_r theta_n = exp(j2pi c (r N_S + S_n)/N))
      const FcSize& zN = P.sz[G.size_N];
      const float2 ph0 = pos_root(zN, (long long)S.c * G.cps[n]);
      const float2 ph1 = pos_root(zN, (long long)S.c * (G.cps[n] + G.N_S));
      tx_map(S, N, Z, Y, ph0, ph1, 2);
    }
    // T6: long IDFTs (1/N and sqrt(I) folded into D)
    fft_inplace<true>(Y, 2, P.sz[G.size_N]);
    // T7: R_N^{(r)} combination (OLS windows s_{m,0}, s_{m,1}), Gamma_sigma placement into the ring
    const int h = N / 2, ncp = G.ncp[n];
    const bool ols = P.scheme_tx == FC_OLS;
    int r = ((jb.start + (int)threadIdx.x) % RS + RS) % RS;
    for (int tau = threadIdx.x; tau < 3 * h; tau += FC_THREADS, r = ring_step(r, RS)) {
      float2 v = make_float2(0.f, 0.f);
      if (tau < N && (!ols || (tau >= G.N_L - ncp && tau < G.N_L + G.N_S))) v = cadd(v, Y[sp(tau)]);
      if (tau >= h) {
        const int t = tau - h;
        if (!ols || (t >= G.N_L && t < G.N_L + G.N_S)) v = cadd(v, Y[sp(N + t)]);
      }
      const int T = jb.start + tau;
      if (T >= flushed && T < ch.t1) ring[r] = cadd(ring[r], v);
    }
    __syncthreads();
    const int upto = (j + 1 < ch.j1) ? min(jobs[j + 1].start, ch.t1) : ch.t1;
    if (upto > flushed) {
      ring_flush(ring, RS, wdst, flushed, upto);
      flushed = upto;
    }
  }
  if (ch.t1 > flushed) ring_flush(ring, RS, wdst, flushed, ch.t1);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_tx_sync(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, const FcChunk* __restrict__ chunks,
          int n_chunks, const TI* __restrict__ grid, TO* __restrict__ wave) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  load_plan(P, gP);
  const int stream = blockIdx.x / n_chunks;
  tx_sync_chunk(P, jobs, chunks[blockIdx.x - stream * n_chunks], stream, grid, wave, smem_raw);
}

// ---------------------------------------------------------------------------
// Symbol-synchronized RX (Sec. IV)
// ---------------------------------------------------------------------------
template <typename TI, typename TO>
__device__ __forceinline__ void rx_sync_chunk(const FcPlanDev& P, const FcJob* __restrict__ jobs, const FcChunk ch,
                                              int stream, const TI* __restrict__ wave, TO* __restrict__ grid,
                                              unsigned char* smem_raw) {
  float2* Y = reinterpret_cast<float2*>(smem_raw);
  float2* W = Y + P.ybuf;
  const TI* src = wave + (size_t)stream * P.frame_len;
  const bool io_time = (P.flags & FC_FLAG_IO_TIME) != 0;
  TO* gdst = grid + (size_t)stream * (io_time ? P.time_rx_len : P.grid_len);
  const bool ola = P.scheme_rx == FC_OLA;

  for (int j = ch.j0; j < ch.j1; ++j) {
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    const int N = G.N, n = jb.index, h = N / 2;
    // R1: segmentation w_hat^{(r)} = (R_N^{(r)})^T Gamma_sigma^T x_hat, high-rate A window for OLA (eq:1)
    for (int idx = threadIdx.x; idx < 2 * N; idx += FC_THREADS) {
      const int r = idx >= N;
      const int t = idx - r * N;
      float2 v = io_ld(src + jb.start + r * h + t);
      if (ola && !(t >= G.N_L && t < G.N_L + G.N_S)) v = make_float2(0.f, 0.f);
      Y[sp(idx)] = v;
    }
    __syncthreads();
    // R2: long DFTs
    fft_inplace<false>(Y, 2, P.sz[G.size_N]);
    for (int m = G.first_sub; m < G.first_sub + G.n_sub; ++m) {
      const FcSubDev& S = P.s[m];
      const int L = S.L, q4 = L / 4;
      const FcSize& zN = P.sz[G.size_N];
      const float2 ph0 = pos_root(zN, (long long)S.c * G.cps[n]);
      const float2 ph1 = pos_root(zN, (long long)S.c * (G.cps[n] + G.N_S));
      // R3: gather with conj(phi_r theta_n), D_m, inverse shift
      rx_gather(S, N, Y, W, ph0, ph1, 2);
      // R4: short IDFTs (1/(sqrt(I) L) folded into D)
      fft_inplace<true>(W, 2, P.sz[S.size_L]);
      // R5: S window and concatenation (eq:concat2), or OLA of the two blocks
      float2* X = W + fc_padded_len(2 * L);
      for (int t = threadIdx.x; t < L; t += FC_THREADS) {
        float2 v;
        if (!ola) {
          v = t < L / 2 ? W[sp(q4 + t)] : W[sp(L + t - q4)];
        } else {
          const int u = q4 + t;
          v = make_float2(0.f, 0.f);
          if (u < L) v = cadd(v, W[sp(u)]);
          if (u >= L / 2) v = cadd(v, W[sp(L + u - L / 2)]);
        }
        X[sp(t)] = v;
        if (io_time) io_st(gdst + S.time_rx_off + (long long)n * L + t, cscale(v, sqrtf((float)S.Lofdm)));   // body, true scale
      }
      __syncthreads();
      if (io_time) continue;
      // R6: OFDM demodulation, active bins out
      fft_inplace<false>(X, 1, P.sz[S.size_O]);
      TO* row = gdst + S.grid_off + (long long)n * S.Lact;
      for (int a = threadIdx.x; a < S.Lact; a += FC_THREADS) {
        int bin = a - S.Lact / 2;
        if (bin < 0) bin += L;
        io_st(row + a, X[sp(bin)]);
      }
      __syncthreads();
    }
  }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_rx_sync(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, const FcChunk* __restrict__ chunks,
          int n_chunks, const TI* __restrict__ wave, TO* __restrict__ grid) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  load_plan(P, gP);
  const int stream = blockIdx.x / n_chunks;
  rx_sync_chunk(P, jobs, chunks[blockIdx.x - stream * n_chunks], stream, wave, grid, smem_raw);
}

// ---------------------------------------------------------------------------
// Symbol-synchronized TX or RX of many plans in one persistent launch: each CTA takes
// the next work item (plan, stream, chunk) from a device counter, reloads its shared
// plan copy only when the plan changes, and runs the chunk. One launch serves items of
// one I/O type T (a queue holds complex64 or complex-BF16 items, never both).
// ---------------------------------------------------------------------------
template <bool TX, typename T>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_sync_multi(const FcWork* __restrict__ work, int n_work, int* __restrict__ next) {
  __shared__ FcPlanDev P;
  __shared__ int item;
  __shared__ const FcPlanDev* loaded;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (threadIdx.x == 0) loaded = nullptr;
  while (true) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int i = item;
    if (i >= n_work) break;
    const FcWork w = work[i];
    if (w.plan != loaded) {
      load_plan(P, w.plan);                     // ends with a barrier
      if (threadIdx.x == 0) loaded = w.plan;
    }
    if (TX)                                     // frame calls: input and output of one type T
      tx_sync_chunk(P, w.jobs, *w.chunk, w.stream, (const T*)w.in, (T*)w.out, smem_raw);
    else
      rx_sync_chunk(P, w.jobs, *w.chunk, w.stream, (const T*)w.in, (T*)w.out, smem_raw);
    __syncthreads();                            // item and the plan copy are reused
  }
}

// ---------------------------------------------------------------------------
// Continuous mode, stage 1 (TX): CP-OFDM symbols -> low-rate stream s_m (workspace)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool locate_symbol(const FcPlanDev& P, int& m, int& n, int per_stream_idx) {
  int acc = 0;
  for (m = 0; m < P.n_subs; ++m) {
    const int B = P.g[P.s[m].group].B;
    if (per_stream_idx < acc + B) {
      n = per_stream_idx - acc;
      return true;
    }
    acc += B;
  }
  return false;
}

template <typename TI>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_ofdm_mod(const FcPlanDev* __restrict__ gP, int syms_per_stream, const TI* __restrict__ grid,
           float2* __restrict__ ws) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  load_plan(P, gP);
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int stream = blockIdx.x / syms_per_stream;
  int m, n;
  if (!locate_symbol(P, m, n, blockIdx.x - stream * syms_per_stream)) return;
  const FcSubDev& S = P.s[m];
  const int L = S.Lofdm, lcp = S.lcp[n];
  float2* dst = ws + (size_t)stream * P.ws_len + S.ws_off + S.soff[n];
  if (P.flags & FC_FLAG_IO_TIME) {       // the caller's CP and body, brought to the kernels' scale
    const TI* src = grid + (size_t)stream * P.time_tx_len + S.time_tx_off + S.soff[n];
    for (int i = threadIdx.x; i < lcp + L; i += FC_THREADS) dst[i] = cscale(io_ld(src + i), sqrtf((float)S.Lofdm));
    return;
  }
  ofdm_symbol_to_time(P, S, grid + (size_t)stream * P.grid_len + S.grid_off + (long long)n * S.Lact, buf);
  for (int i = threadIdx.x; i < lcp + L; i += FC_THREADS) {   // K_{L_CP} (eq:TX_CPins)
    int bi = i - lcp;
    if (bi < 0) bi += L;
    dst[i] = buf[sp(bi)];
  }
}

// ---------------------------------------------------------------------------
// Continuous mode, stage 2 (TX): FC blocks over [0_{S_L}; s; 0_{S_L}] (eq:BDM)
// ---------------------------------------------------------------------------
template <typename TO>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_tx_cont(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, const FcChunk* __restrict__ chunks,
          int n_chunks, const float2* __restrict__ ws, TO* __restrict__ wave) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  load_plan(P, gP);
  float2* ring = reinterpret_cast<float2*>(smem_raw);
  float2* Y = ring + P.ring;
  float2* Z = Y + P.ybuf;
  const int stream = blockIdx.x / n_chunks;
  const FcChunk ch = chunks[blockIdx.x - stream * n_chunks];
  const float2* wsrc = ws + (size_t)stream * P.ws_len;
  TO* wdst = wave + (size_t)stream * P.frame_len;
  const int RS = P.ring;
  const bool ols = P.scheme_tx == FC_OLS;
  zero_buf(ring, RS);
  int flushed = ch.t0;
  __syncthreads();

  for (int j = ch.j0; j < ch.j1; ++j) {
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    const int N = G.N, r0 = jb.index, nb = jb.nblk;
    zero_buf(Y, fc_padded_len(2 * N));
    __syncthreads();
    for (int m = G.first_sub; m < G.first_sub + G.n_sub; ++m) {
      const FcSubDev& S = P.s[m];
      const int L = S.L;
      const float2* s = wsrc + S.ws_off;
      // segmentation, A_{m,r} for OLA (eq:ola_proc)
      for (int idx = threadIdx.x; idx < 2 * L; idx += FC_THREADS) {
        const int b = idx >= L;
        const int t = idx - b * L;
        const int pos = (r0 + b) * S.L_S + t - S.S_L;
        float2 v = make_float2(0.f, 0.f);
        if (b < nb && pos >= 0 && pos < S.n_low && (ols || (t >= S.L_L && t < S.L_L + S.L_S))) v = __ldg(s + pos);
        Z[sp(idx)] = v;
      }
      __syncthreads();
      fft_inplace<false>(Z, 2, P.sz[S.size_L]);
      const FcSize& zN = P.sz[G.size_N];
      const float2 ph0 = pos_root(zN, (long long)S.c * r0 * G.N_S);         // phi_{m,r}
      const float2 ph1 = pos_root(zN, (long long)S.c * (r0 + 1) * G.N_S);
      tx_map(S, N, Z, Y, ph0, ph1, nb);
    }
    fft_inplace<true>(Y, 2, P.sz[G.size_N]);
    // OLA accumulate / OLS discard (S_{m,r}) into the ring
    const int span = G.N_S + N;
    int r = ((jb.start + (int)threadIdx.x) % RS + RS) % RS;
    for (int tau = threadIdx.x; tau < span; tau += FC_THREADS, r = ring_step(r, RS)) {
      float2 v = make_float2(0.f, 0.f);
      if (tau < N && (!ols || (tau >= G.N_L && tau < G.N_L + G.N_S))) v = cadd(v, Y[sp(tau)]);
      if (nb > 1 && tau >= G.N_S) {
        const int t = tau - G.N_S;
        if (!ols || (t >= G.N_L && t < G.N_L + G.N_S)) v = cadd(v, Y[sp(N + t)]);
      }
      const int T = jb.start + tau;
      if (T >= flushed && T < ch.t1) ring[r] = cadd(ring[r], v);
    }
    __syncthreads();
    const int upto = (j + 1 < ch.j1) ? min(jobs[j + 1].start, ch.t1) : ch.t1;
    if (upto > flushed) {
      ring_flush(ring, RS, wdst, flushed, upto);
      flushed = upto;
    }
  }
  if (ch.t1 > flushed) ring_flush(ring, RS, wdst, flushed, ch.t1);
}

// ---------------------------------------------------------------------------
// Continuous mode, stage 1 (RX): FC analysis blocks -> low-rate stream (OLS,
// disjoint kept parts) or per-block outputs (OLA, summed by the demodulator)
// ---------------------------------------------------------------------------
template <typename TI>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_rx_cont(const FcPlanDev* __restrict__ gP, const FcJob* __restrict__ jobs, const FcChunk* __restrict__ chunks,
          int n_chunks, const TI* __restrict__ wave, float2* __restrict__ ws) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  load_plan(P, gP);
  float2* Y = reinterpret_cast<float2*>(smem_raw);
  float2* V = Y + P.ybuf;
  const int stream = blockIdx.x / n_chunks;
  const FcChunk ch = chunks[blockIdx.x - stream * n_chunks];
  const TI* src = wave + (size_t)stream * P.frame_len;
  float2* wdst = ws + (size_t)stream * P.ws_len;
  const bool ola = P.scheme_rx == FC_OLA;

  for (int j = ch.j0; j < ch.j1; ++j) {
    const FcJob jb = jobs[j];
    const FcGroupDev& G = P.g[jb.group];
    const int N = G.N, r0 = jb.index, nb = jb.nblk;
    for (int idx = threadIdx.x; idx < 2 * N; idx += FC_THREADS) {
      const int b = idx >= N;
      const int t = idx - b * N;
      float2 v = make_float2(0.f, 0.f);
      if (b < nb && (!ola || (t >= G.N_L && t < G.N_L + G.N_S))) v = io_ld(src + jb.start + b * G.N_S + t);
      Y[sp(idx)] = v;
    }
    __syncthreads();
    fft_inplace<false>(Y, 2, P.sz[G.size_N]);
    for (int m = G.first_sub; m < G.first_sub + G.n_sub; ++m) {
      const FcSubDev& S = P.s[m];
      const int L = S.L;
      const FcSize& zN = P.sz[G.size_N];
      const float2 ph0 = pos_root(zN, (long long)S.c * r0 * G.N_S);
      const float2 ph1 = pos_root(zN, (long long)S.c * (r0 + 1) * G.N_S);
      rx_gather(S, N, Y, V, ph0, ph1, nb);
      fft_inplace<true>(V, 2, P.sz[S.size_L]);
      float2* d = wdst + S.ws_off;
      if (!ola) {   // S_{m,r}: keep [L_L, L_L + L_S) at low-rate position r L_S + L_L
        for (int idx = threadIdx.x; idx < nb * S.L_S; idx += FC_THREADS) {
          const int b = idx >= S.L_S;
          const int t = S.L_L + idx - b * S.L_S;
          const int pos = (r0 + b) * S.L_S + t - S.S_L;
          if (pos >= 0 && pos < S.n_low) d[pos] = V[sp(b * L + t)];
        }
      } else {      // keep whole blocks; overlapping parts are added by the demodulator
        for (int idx = threadIdx.x; idx < nb * L; idx += FC_THREADS) {
          const int b = idx >= L;
          d[(long long)(r0 + b) * L + idx - b * L] = V[sp(idx)];
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Continuous mode, stage 2 (RX): CP removal and OFDM demodulation
// ---------------------------------------------------------------------------
template <typename TO>
__global__ void __launch_bounds__(FC_THREADS, FC_GEN_MIN_BLOCKS)
k_ofdm_demod(const FcPlanDev* __restrict__ gP, int syms_per_stream, const float2* __restrict__ ws,
             TO* __restrict__ grid) {
  __shared__ FcPlanDev P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  load_plan(P, gP);
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int stream = blockIdx.x / syms_per_stream;
  int m, n;
  if (!locate_symbol(P, m, n, blockIdx.x - stream * syms_per_stream)) return;
  const FcSubDev& S = P.s[m];
  const FcGroupDev& G = P.g[S.group];
  const float2* s = ws + (size_t)stream * P.ws_len + S.ws_off;
  const int Lo = S.Lofdm, base = S.soff[n] + S.lcp[n];
  const bool ola = P.scheme_rx == FC_OLA;
  for (int t = threadIdx.x; t < Lo; t += FC_THREADS) {
    float2 v = make_float2(0.f, 0.f);
    if (!ola) {
      v = __ldg(s + base + t);
    } else {
      const int Pu = S.S_L + base + t;                       // position in the padded stream
      int r_hi = Pu / S.L_S;
      if (r_hi > G.R - 1) r_hi = G.R - 1;
      for (int r = r_hi; r >= 0 && Pu - r * S.L_S < S.L; --r) v = cadd(v, __ldg(s + (long long)r * S.L + Pu - r * S.L_S));
    }
    buf[sp(t)] = v;
    if (P.flags & FC_FLAG_IO_TIME)       // the body before demodulation, true scale
      io_st(grid + (size_t)stream * P.time_rx_len + S.time_rx_off + (long long)n * Lo + t, cscale(v, sqrtf((float)S.Lofdm)));
  }
  if (P.flags & FC_FLAG_IO_TIME) return;
  __syncthreads();
  fft_inplace<false>(buf, 1, P.sz[S.size_O]);
  TO* row = grid + (size_t)stream * P.grid_len + S.grid_off + (long long)n * S.Lact;
  for (int a = threadIdx.x; a < S.Lact; a += FC_THREADS) {
    int bin = a - S.Lact / 2;
    if (bin < 0) bin += Lo;
    io_st(row + a, buf[sp(bin)]);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers (file-local; exported as this compilation's FcGenKernels table)
// ---------------------------------------------------------------------------
namespace {
template <bool TX, typename T>
cudaError_t launch_multi(const FcWork* work, int n_work, int* next, int num_sms, size_t smem, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sync_multi<TX, T>, FC_THREADS, smem);
  if (e != cudaSuccess) return e;
  int n_ctas = num_sms * (per_sm > 0 ? per_sm : 1);
  if (n_ctas > n_work) n_ctas = n_work;
  k_sync_multi<TX, T><<<n_ctas, FC_THREADS, smem, st>>>(work, n_work, next);
  return cudaGetLastError();
}

cudaError_t launch_sync_multi(bool tx, const FcWork* work, int n_work, int io, int* next, int num_sms, size_t smem,
                                 cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(int), st);
  if (e != cudaSuccess || n_work == 0) return e;
  if (io != 0 && io != (FC_IO_IN_BF16 | FC_IO_OUT_BF16)) return cudaErrorInvalidValue;
  if (tx)
    return io ? launch_multi<true, bf2>(work, n_work, next, num_sms, smem, st)
              : launch_multi<true, float2>(work, n_work, next, num_sms, smem, st);
  return io ? launch_multi<false, bf2>(work, n_work, next, num_sms, smem, st)
            : launch_multi<false, float2>(work, n_work, next, num_sms, smem, st);
}

cudaError_t launch_tx_sync(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks,
                              int n_streams, const void* grid, void* wave, int io, size_t smem, cudaStream_t st) {
  const dim3 g((unsigned)(n_streams * n_chunks));
  if (io == 0)
    k_tx_sync<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const float2*)grid, (float2*)wave);
  else if (io == (FC_IO_IN_BF16 | FC_IO_OUT_BF16))
    k_tx_sync<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const bf2*)grid, (bf2*)wave);
  else if (io == FC_IO_IN_BF16)
    k_tx_sync<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const bf2*)grid, (float2*)wave);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_rx_sync(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks,
                              int n_streams, const void* wave, void* grid, int io, size_t smem, cudaStream_t st) {
  const dim3 g((unsigned)(n_streams * n_chunks));
  if (io == 0)
    k_rx_sync<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const float2*)wave, (float2*)grid);
  else if (io == (FC_IO_IN_BF16 | FC_IO_OUT_BF16))
    k_rx_sync<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const bf2*)wave, (bf2*)grid);
  else if (io == FC_IO_OUT_BF16)
    k_rx_sync<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const float2*)wave, (bf2*)grid);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_ofdm_mod(const FcPlanDev* dP, int syms_per_stream, int n_streams, const void* grid,
                               float2* ws, int io, size_t smem, cudaStream_t st) {
  const dim3 g((unsigned)(n_streams * syms_per_stream));
  if (io & FC_IO_IN_BF16)
    k_ofdm_mod<<<g, FC_THREADS, smem, st>>>(dP, syms_per_stream, (const bf2*)grid, ws);
  else
    k_ofdm_mod<<<g, FC_THREADS, smem, st>>>(dP, syms_per_stream, (const float2*)grid, ws);
  return cudaGetLastError();
}

cudaError_t launch_tx_cont(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks,
                              int n_streams, const float2* ws, void* wave, int io, size_t smem, cudaStream_t st) {
  const dim3 g((unsigned)(n_streams * n_chunks));
  if (io & FC_IO_OUT_BF16)
    k_tx_cont<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, ws, (bf2*)wave);
  else
    k_tx_cont<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, ws, (float2*)wave);
  return cudaGetLastError();
}

cudaError_t launch_rx_cont(const FcPlanDev* dP, const FcJob* jobs, const FcChunk* chunks, int n_chunks,
                              int n_streams, const void* wave, float2* ws, int io, size_t smem, cudaStream_t st) {
  const dim3 g((unsigned)(n_streams * n_chunks));
  if (io & FC_IO_IN_BF16)
    k_rx_cont<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const bf2*)wave, ws);
  else
    k_rx_cont<<<g, FC_THREADS, smem, st>>>(dP, jobs, chunks, n_chunks, (const float2*)wave, ws);
  return cudaGetLastError();
}

cudaError_t launch_ofdm_demod(const FcPlanDev* dP, int syms_per_stream, int n_streams, const float2* ws,
                                 void* grid, int io, size_t smem, cudaStream_t st) {
  const dim3 g((unsigned)(n_streams * syms_per_stream));
  if (io & FC_IO_OUT_BF16)
    k_ofdm_demod<<<g, FC_THREADS, smem, st>>>(dP, syms_per_stream, ws, (bf2*)grid);
  else
    k_ofdm_demod<<<g, FC_THREADS, smem, st>>>(dP, syms_per_stream, ws, (float2*)grid);
  return cudaGetLastError();
}

template <typename K>
cudaError_t raise_smem(K kernel, size_t max_smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
}

cudaError_t set_smem_limits(size_t max_smem) {
  const cudaError_t e[] = {
      raise_smem(k_tx_sync<float2, float2>, max_smem), raise_smem(k_tx_sync<bf2, bf2>, max_smem),
      raise_smem(k_tx_sync<bf2, float2>, max_smem),    raise_smem(k_rx_sync<float2, float2>, max_smem),
      raise_smem(k_rx_sync<bf2, bf2>, max_smem),       raise_smem(k_rx_sync<float2, bf2>, max_smem),
      raise_smem(k_sync_multi<true, float2>, max_smem), raise_smem(k_sync_multi<false, float2>, max_smem),
      raise_smem(k_sync_multi<true, bf2>, max_smem),    raise_smem(k_sync_multi<false, bf2>, max_smem),
      raise_smem(k_tx_cont<float2>, max_smem),         raise_smem(k_tx_cont<bf2>, max_smem),
      raise_smem(k_rx_cont<float2>, max_smem),         raise_smem(k_rx_cont<bf2>, max_smem),
      raise_smem(k_ofdm_mod<float2>, max_smem),        raise_smem(k_ofdm_mod<bf2>, max_smem),
      raise_smem(k_ofdm_demod<float2>, max_smem),      raise_smem(k_ofdm_demod<bf2>, max_smem)};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}
}  // namespace

#define FC_GEN_CAT2(a, b) a##b
#define FC_GEN_CAT(a, b) FC_GEN_CAT2(a, b)
const FcGenKernels& FC_GEN_CAT(fc_gen_kernels_, FC_THREADS)() {
  static const FcGenKernels k{FC_THREADS,  launch_sync_multi, launch_tx_sync,   launch_rx_sync, launch_ofdm_mod,
                              launch_tx_cont, launch_rx_cont,  launch_ofdm_demod, set_smem_limits};
  return k;
}

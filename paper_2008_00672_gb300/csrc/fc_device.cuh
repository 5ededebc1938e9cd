// Device helpers shared by the FC kernels: complex arithmetic, multiplication by
// the 32nd roots of unity with compile-time constants, and in-register DFTs of
// 2..32 points (natural order in and out). Forward = exp(-j...), inverse =
// exp(+j...) without the 1/n factor.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace fcdev {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// multiply by -j (forward) or +j (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mj(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi m / 32) for m in [0, 32): first-octant values and symmetries
__host__ __device__ constexpr float c32_base(int m) {
  return m == 0 ? 1.0f
       : m == 1 ? 0.98078528040323044913f
       : m == 2 ? 0.92387953251128675613f
       : m == 3 ? 0.83146961230254523708f
       : m == 4 ? 0.70710678118654752440f
       : m == 5 ? 0.55557023301960222474f
       : m == 6 ? 0.38268343236508977173f
       : m == 7 ? 0.19509032201612826785f
                : 0.0f;
}
__host__ __device__ constexpr float c32(int m) {
  return m > 16 ? c32(32 - m) : (m > 8 ? -c32_base(16 - m) : c32_base(m));
}
// sin(2 pi m / 32)
__host__ __device__ constexpr float s32(int m) { return c32((m + 24) & 31); }

// a * W_32^{M} (forward: exp(-j 2 pi M/32); inverse: exp(+j 2 pi M/32))
template <int M, bool INV>
__device__ __forceinline__ float2 tw32(float2 a) {
  constexpr int m = M & 31;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 8) {
    return mul_mj<INV>(a);
  } else if constexpr (m == 16) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (m == 24) {
    return mul_mj<!INV>(a);
  } else {
    constexpr float c = c32(m);
    constexpr float s = s32(m);
    if constexpr (INV) return make_float2(a.x * c - a.y * s, a.y * c + a.x * s);
    else return make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
  }
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = mul_mj<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// In-register DFT of R points on v[0..R), natural order in and out.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <bool INV>
struct Dft<3, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float s = 0.86602540378443864676f;   // sin(2 pi/3); cos(2 pi/3) = -1/2
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
  static __device__ __forceinline__ void run(float2* v) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};

// R = R1 x R2 with R1 = 2 (inner, stride R2) and R2 in {4, 8, 16}:
//   X[k1 + 2 k2] = sum_t2 W_R2^{t2 k2} W_R^{t2 k1} sum_t1 x[t2 + R2 t1] W_2^{t1 k1}
template <int R, bool INV>
struct DftSplit2 {
  static constexpr int H = R / 2;
  static __device__ __forceinline__ void run(float2* v) {
#pragma unroll
    for (int t2 = 0; t2 < H; ++t2) {
      const float2 a = v[t2];
      v[t2] = cadd(a, v[t2 + H]);
      v[t2 + H] = csub(a, v[t2 + H]);
    }
    twiddle_odd(v + H, std::integral_constant<int, 1>());
    Dft<H, INV>::run(v);
    Dft<H, INV>::run(v + H);
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = t[(k & 1) * H + (k >> 1)];
  }
  // v[t2] *= W_R^{t2} for t2 = 1..H-1 (W_R^{t2} = W_32^{t2 * 32/R})
  template <int T2>
  static __device__ __forceinline__ void twiddle_odd(float2* v, std::integral_constant<int, T2>) {
    if constexpr (T2 < H) {
      v[T2] = tw32<T2 * (32 / R), INV>(v[T2]);
      twiddle_odd(v, std::integral_constant<int, T2 + 1>());
    }
  }
};

template <bool INV>
struct Dft<8, INV> {
  static __device__ __forceinline__ void run(float2* v) { DftSplit2<8, INV>::run(v); }
};

// 16 = 4 x 4: inner 4-point DFTs over t1 (stride 4), twiddle W_16^{t2 k1}, outer 4-point DFTs.
template <bool INV>
struct Dft<16, INV> {
  static __device__ __forceinline__ void run(float2* v) {
#pragma unroll
    for (int t2 = 0; t2 < 4; ++t2) dft4<INV>(v[t2], v[t2 + 4], v[t2 + 8], v[t2 + 12]);
    v[5] = tw32<2, INV>(v[5]);
    v[6] = tw32<4, INV>(v[6]);
    v[7] = tw32<6, INV>(v[7]);
    v[9] = tw32<4, INV>(v[9]);
    v[10] = tw32<8, INV>(v[10]);
    v[11] = tw32<12, INV>(v[11]);
    v[13] = tw32<6, INV>(v[13]);
    v[14] = tw32<12, INV>(v[14]);
    v[15] = tw32<18, INV>(v[15]);
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

template <bool INV>
struct Dft<32, INV> {
  static __device__ __forceinline__ void run(float2* v) { DftSplit2<32, INV>::run(v); }
};

}  // namespace fcdev

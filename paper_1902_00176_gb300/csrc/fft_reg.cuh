// fft_reg.cuh -- compile-time register DFTs of composite length (device side).
//
// dft_reg<R, DIR>(v) replaces v[0..R) by V[k] = sum_m v[m] w^(m k),
// w = exp(DIR 2 pi i / R), in natural order, entirely in registers. A
// composite R = A B is split by Cooley-Tukey decimation in time:
//   Y_a[k1] = sum_b v[a + A b] w_B^(b k1)          (A transforms of length B)
//   V[k1 + B k2] = sum_a (w_R^(a k1) Y_a[k1]) w_A^(a k2)   (B transforms of length A)
// and recursed until the base radices 2, 3, 4, 5, 7, 8 (fft_core.cuh). The
// inner twiddles w_R^(a k1) are compile-time constants: trivial ones (1, -1,
// +-i, (+-1 +-i)/sqrt 2) become adds/sign swaps, the rest a complex multiply
// by constants computed at compile time from the Taylor series of sin and cos.
#pragma once

#include "fft_core.cuh"

namespace gfc {

// ---- compile-time sin/cos of 2 pi e / R (Taylor series on [-pi/4, pi/4]) ----
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double cx_taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double cx_taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi e / R for integers 0 <= e < R, by octant reduction on
// the exact integer fraction (8 e) / R before any rounding.
constexpr double cx_cos2pi(long e, long R) {
  e %= R;
  if (e < 0) e += R;
  // angle in units of pi/4: q = 8 e / R; reduce by the octant index
  const long o = (8 * e) / R;                              // octant 0..7
  const double f = (double)(8 * e - o * R) / (double)R;    // in [0, 1)
  const double x = f * (kPi / 4.0);
  switch (o) {
    case 0: return cx_taylor_cos(x);
    case 1: return cx_taylor_sin(kPi / 4.0 - x);
    case 2: return -cx_taylor_sin(x);
    case 3: return -cx_taylor_cos(kPi / 4.0 - x);
    case 4: return -cx_taylor_cos(x);
    case 5: return -cx_taylor_sin(kPi / 4.0 - x);
    case 6: return cx_taylor_sin(x);
    default: return cx_taylor_cos(kPi / 4.0 - x);
  }
}
constexpr double cx_sin2pi(long e, long R) {
  e %= R;
  if (e < 0) e += R;
  const long o = (8 * e) / R;
  const double f = (double)(8 * e - o * R) / (double)R;
  const double x = f * (kPi / 4.0);
  switch (o) {
    case 0: return cx_taylor_sin(x);
    case 1: return cx_taylor_cos(kPi / 4.0 - x);
    case 2: return cx_taylor_cos(x);
    case 3: return cx_taylor_sin(kPi / 4.0 - x);
    case 4: return -cx_taylor_sin(x);
    case 5: return -cx_taylor_cos(kPi / 4.0 - x);
    case 6: return -cx_taylor_cos(x);
    default: return -cx_taylor_sin(kPi / 4.0 - x);
  }
}

// x * w_R^e with w_R = exp(DIR 2 pi i / R), e a compile-time integer
template <int R, int E, int DIR>
__device__ __forceinline__ float2 twc(float2 x) {
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return x;
  } else if constexpr (2 * e == R) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (4 * e == R) {
    return rot<DIR>(x);  // w = DIR i
  } else if constexpr (4 * e == 3 * R) {
    return rot<-DIR>(x);  // w = -DIR i
  } else if constexpr (8 * e == R || 8 * e == 3 * R || 8 * e == 5 * R || 8 * e == 7 * R) {
    constexpr float h = 0.707106781186547524401f;
    constexpr int oct = (8 * e) / R;  // 1, 3, 5, 7
    // w = (cx + DIR i sx) / sqrt2 with cx, sx in {+-1}
    constexpr float cx = (oct == 1 || oct == 7) ? 1.0f : -1.0f;
    constexpr float sx = (oct == 1 || oct == 3) ? 1.0f : -1.0f;
    const float2 r = rot<DIR>(x);  // x * DIR i
    return make_float2(h * (cx * x.x + sx * r.x), h * (cx * x.y + sx * r.y));
  } else {
    constexpr float c = (float)cx_cos2pi(e, R);
    constexpr float s = (float)(DIR * cx_sin2pi(e, R));
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
  }
}

constexpr bool is_base_radix(int R) { return R == 2 || R == 3 || R == 4 || R == 5 || R == 7 || R == 8; }

// first factor A of a composite R (the length of the outer transforms): the
// largest base radix not above sqrt(R), which keeps the temporaries of each
// sub-transform small (register pressure), else the smallest prime factor
constexpr int split_factor(int R) {
  int best = 0;
  for (int f : {2, 3, 4, 5, 7, 8})
    if (R % f == 0 && f * f <= R && f > best) best = f;
  if (best) return best;
  for (int f : {2, 3, 5, 7})
    if (R % f == 0) return f;
  return R;
}

template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2* v);

template <int R, int DIR, int A, int B, int K1>
__device__ __forceinline__ void dft_reg_twiddle_row(float2 (&t)[R]) {
  // t[a B + K1] *= w_R^(a K1) for a < A
  [&]<int... a>(std::integer_sequence<int, a...>) {
    ((t[a * B + K1] = twc<R, a * K1, DIR>(t[a * B + K1])), ...);
  }(std::make_integer_sequence<int, A>{});
}

template <int R, int DIR, int A, int B>
__device__ __forceinline__ void dft_reg_split(float2* v) {
  float2 t[R];
#pragma unroll
  for (int a = 0; a < A; ++a) {
    float2 s[B];
#pragma unroll
    for (int b = 0; b < B; ++b) s[b] = v[a + A * b];
    dft_reg<B, DIR>(s);
#pragma unroll
    for (int k = 0; k < B; ++k) t[a * B + k] = s[k];
  }
  [&]<int... k1>(std::integer_sequence<int, k1...>) {
    (dft_reg_twiddle_row<R, DIR, A, B, k1>(t), ...);
  }(std::make_integer_sequence<int, B>{});
#pragma unroll
  for (int k1 = 0; k1 < B; ++k1) {
    float2 s[A];
#pragma unroll
    for (int a = 0; a < A; ++a) s[a] = t[a * B + k1];
    dft_reg<A, DIR>(s);
#pragma unroll
    for (int k2 = 0; k2 < A; ++k2) v[k1 + B * k2] = s[k2];
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (is_base_radix(R)) {
    dft<R, DIR>(v);
  } else {
    constexpr int A = split_factor(R);
    static_assert(A != R, "dft_reg: R must be 7-smooth");
    dft_reg_split<R, DIR, A, R / A>(v);
  }
}

}  // namespace gfc

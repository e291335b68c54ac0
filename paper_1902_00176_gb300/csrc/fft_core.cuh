// fft_core.cuh -- mixed-radix Stockham FFT building blocks (device side).
//
// The transform is the DFT of Eq. 17 (X[k] = sum_m x[m] w^(k m), w = exp(DIR 2 pi i / n),
// DIR = -1 forward, +1 unnormalised inverse), computed by the Stockham
// autosort formulation of Cooley-Tukey: a sequence of radix-R stages with
// span Ns (product of the radices before the stage). Stage (R, Ns) maps
// butterfly j in [0, n/R), k = j mod Ns:
//     v[r]  = in[j + r n/R] * w_(Ns R)^(r k)                    r < R
//     V     = DFT_R(v)
//     out[(j div Ns) Ns R + k + s Ns] = V[s]                    s < R
// Input and output are in natural order. Twiddles come from one table of the
// n-th roots of unity, tw[m] = exp(-2 pi i m / n), built in FP64 and rounded
// once; w_(Ns R)^(r k) = tw[r k n / (Ns R)] (the inverse uses the conjugate).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gfc {

constexpr int kMaxRadix = 8;
constexpr int kMaxStages = 16;
constexpr int kMaxFftLen = 4096;

struct FftPlan {
  int n;                 // transform length
  int nst;               // number of stages
  int radix[kMaxStages]; // radix of each stage, in order
};

// Complex helpers. Component-wise pair operations use the packed FP32
// instructions of sm_100+ (one instruction for both halves, same rounding as
// two scalar ones); operations that swap the halves stay scalar.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): exact negation, one rounding, identical to a - b
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// a * s + c
__device__ __forceinline__ float2 cfma(float2 a, float s, float2 c) { return __ffma2_rn(a, make_float2(s, s), c); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * (DIR i): DIR = -1 gives a * (-i) = (a.y, -a.x); DIR = +1 gives (-a.y, a.x).
template <int DIR>
__device__ __forceinline__ float2 rot(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
// p + rot(q) and p - rot(q)
template <int DIR>
__device__ __forceinline__ float2 add_rot(float2 p, float2 q) {
  return DIR < 0 ? make_float2(p.x + q.y, p.y - q.x) : make_float2(p.x - q.y, p.y + q.x);
}
template <int DIR>
__device__ __forceinline__ float2 sub_rot(float2 p, float2 q) {
  return DIR < 0 ? make_float2(p.x - q.y, p.y + q.x) : make_float2(p.x + q.y, p.y - q.x);
}
// p + s rot(d) and p - s rot(d)
template <int DIR>
__device__ __forceinline__ float2 fma_rot(float2 d, float s, float2 p) {
  return DIR < 0 ? make_float2(fmaf(s, d.y, p.x), fmaf(-s, d.x, p.y)) : make_float2(fmaf(-s, d.y, p.x), fmaf(s, d.x, p.y));
}
// twiddle for direction DIR from a forward-root table value
template <int DIR>
__device__ __forceinline__ float2 tw_dir(float2 w) { return DIR < 0 ? w : cconj(w); }

// ---------------------------------------------------------------------------
// DFT_R butterflies on a register array, V[s] = sum_r v[r] exp(DIR 2 pi i r s / R).
// The odd radices use the symmetric-pair form: with a_m = v_m + v_(R-m),
// b_m = v_m - v_(R-m),
//   V_k     = v_0 + sum_m cos(2 pi k m/R) a_m + DIR i sum_m sin(2 pi k m/R) b_m
//   V_(R-k) = v_0 + sum_m cos(2 pi k m/R) a_m - DIR i sum_m sin(2 pi k m/R) b_m.
// The constants are cos and sin of 2 pi k / R to 21 digits.
// ---------------------------------------------------------------------------

template <int DIR>
__device__ __forceinline__ void dft2(float2* v) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* v) {
  const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  const float2 c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = add_rot<DIR>(b, d);
  v[3] = sub_rot<DIR>(b, d);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
  constexpr float h = 0.707106781186547524401f;  // sqrt(1/2)
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<DIR>(e);
  dft4<DIR>(o);
  // o[s] *= w8^s, w8 = (1 + DIR i) sqrt(1/2); o[2] *= DIR i is folded into the output sums
  const float2 o1 = cscale(add_rot<DIR>(o[1], o[1]), h);
  const float2 o3 = cscale(add_rot<DIR>(make_float2(-o[3].x, -o[3].y), o[3]), h);  // (rot(o3) - o3) / sqrt 2
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = add_rot<DIR>(e[2], o[2]);
  v[6] = sub_rot<DIR>(e[2], o[2]);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

template <int DIR>
__device__ __forceinline__ void dft3(float2* v) {
  constexpr float s60 = 0.866025403784438646764f;
  const float2 t1 = cadd(v[1], v[2]);
  const float2 t2 = cfma(t1, -0.5f, v[0]);
  const float2 d = csub(v[1], v[2]);
  v[0] = cadd(v[0], t1);
  v[1] = fma_rot<DIR>(d, s60, t2);
  v[2] = fma_rot<DIR>(d, -s60, t2);
}

template <int DIR>
__device__ __forceinline__ void dft5(float2* v) {
  constexpr float c1 = 0.309016994374947424102f, c2 = -0.809016994374947424102f;
  constexpr float s1 = 0.951056516295153572116f, s2 = 0.587785252292473129169f;
  const float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
  const float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
  const float2 x0 = v[0];
  const float2 p1 = cfma(a1, c1, cfma(a2, c2, x0));
  const float2 p2 = cfma(a1, c2, cfma(a2, c1, x0));
  const float2 q1 = cfma(b1, s1, cscale(b2, s2));
  const float2 q2 = cfma(b1, s2, cscale(b2, -s1));
  v[0] = cadd(x0, cadd(a1, a2));
  v[1] = add_rot<DIR>(p1, q1);
  v[4] = sub_rot<DIR>(p1, q1);
  v[2] = add_rot<DIR>(p2, q2);
  v[3] = sub_rot<DIR>(p2, q2);
}

template <int DIR>
__device__ __forceinline__ void dft7(float2* v) {
  constexpr float c1 = 0.623489801858733530525f, c2 = -0.222520933956314404289f,
                  c3 = -0.900968867902419126236f;
  constexpr float s1 = 0.781831482468029808708f, s2 = 0.974927912181823607018f,
                  s3 = 0.433883739117558120476f;
  const float2 a1 = cadd(v[1], v[6]), b1 = csub(v[1], v[6]);
  const float2 a2 = cadd(v[2], v[5]), b2 = csub(v[2], v[5]);
  const float2 a3 = cadd(v[3], v[4]), b3 = csub(v[3], v[4]);
  const float2 x0 = v[0];
  // k = 1: (c1, c2, c3), (s1, s2, s3); k = 2: (c2, c3, c1), (s2, -s3, -s1);
  // k = 3: (c3, c1, c2), (s3, -s1, s2)   [cos/sin of 2 pi (k m mod 7)/7]
  const float2 p1 = cfma(a1, c1, cfma(a2, c2, cfma(a3, c3, x0)));
  const float2 p2 = cfma(a1, c2, cfma(a2, c3, cfma(a3, c1, x0)));
  const float2 p3 = cfma(a1, c3, cfma(a2, c1, cfma(a3, c2, x0)));
  const float2 q1 = cfma(b1, s1, cfma(b2, s2, cscale(b3, s3)));
  const float2 q2 = cfma(b1, s2, cfma(b2, -s3, cscale(b3, -s1)));
  const float2 q3 = cfma(b1, s3, cfma(b2, -s1, cscale(b3, s2)));
  v[0] = cadd(x0, cadd(a1, cadd(a2, a3)));
  v[1] = add_rot<DIR>(p1, q1);
  v[6] = sub_rot<DIR>(p1, q1);
  v[2] = add_rot<DIR>(p2, q2);
  v[5] = sub_rot<DIR>(p2, q2);
  v[3] = add_rot<DIR>(p3, q3);
  v[4] = sub_rot<DIR>(p3, q3);
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<DIR>(v);
  else if constexpr (R == 3) dft3<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v);
  else if constexpr (R == 5) dft5<DIR>(v);
  else if constexpr (R == 7) dft7<DIR>(v);
  else if constexpr (R == 8) dft8<DIR>(v);
}

// One Stockham stage of compile-time radix R over `nfft` interleaved
// transforms held in shared memory: element m of transform f lives at
// in[m * es + f]. Threads take (f, j) pairs with f fastest, so a warp reads
// consecutive addresses when es == nfft.
template <int R, int DIR>
__device__ __forceinline__ void stage_smem(const float2* __restrict__ in, float2* __restrict__ out, int n, int Ns,
                                           int nfft, int es, const float2* __restrict__ tw, int tid,
                                           int nthr) {
  const int nb = n / R;
  const int total = nb * nfft;
  const int tstep = n / (Ns * R);
  for (int t = tid; t < total; t += nthr) {
    const int f = t % nfft;
    const int j = t / nfft;
    const int k = j % Ns;
    const int g = j / Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[(j + r * nb) * es + f];
    if (Ns > 1) {
      const int kt = k * tstep;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_dir<DIR>(tw[r * kt]));
    }
    dft<R, DIR>(v);
    const int base = g * Ns * R + k;
#pragma unroll
    for (int s = 0; s < R; ++s) out[(base + s * Ns) * es + f] = v[s];
  }
}

// Run all stages of `pl` on nfft interleaved transforms (layout as above),
// ping-ponging between buf0 and buf1. Returns the buffer holding the result.
// Callers must __syncthreads() before (data in buf0) and after.
template <int DIR>
__device__ float2* fft_smem(float2* buf0, float2* buf1, const FftPlan& pl, int nfft, int es,
                            const float2* __restrict__ tw, int tid, int nthr) {
  float2* a = buf0;
  float2* b = buf1;
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: stage_smem<2, DIR>(a, b, pl.n, Ns, nfft, es, tw, tid, nthr); break;
      case 3: stage_smem<3, DIR>(a, b, pl.n, Ns, nfft, es, tw, tid, nthr); break;
      case 4: stage_smem<4, DIR>(a, b, pl.n, Ns, nfft, es, tw, tid, nthr); break;
      case 5: stage_smem<5, DIR>(a, b, pl.n, Ns, nfft, es, tw, tid, nthr); break;
      case 7: stage_smem<7, DIR>(a, b, pl.n, Ns, nfft, es, tw, tid, nthr); break;
      default: stage_smem<8, DIR>(a, b, pl.n, Ns, nfft, es, tw, tid, nthr); break;
    }
    __syncthreads();
    Ns *= R;
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace gfc

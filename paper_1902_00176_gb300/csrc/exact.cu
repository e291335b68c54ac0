// exact.cu -- solves on Algorithm A's exact padded size (size policy EXACT):
// M = H + 2p, N = W + 2p, whatever their prime factors (801x1200 -> 809x1208,
// where 809 is prime and 1208 = 8 x 151).
//
// Two fields are carried as one complex M x N torus (one Laplacian in the real
// part, the next in the imaginary part): row DFTs of length N, a tiled transpose, column DFTs of
// length M with the Green multiply (Eq. 23) between the forward and the
// inverse transform, a transpose back, inverse row DFTs, then Algorithm B's
// offset and crop. A length that is 7-smooth runs the shared-memory Stockham
// engine directly; any other length n runs Bluestein's chirp-z identity
//     X[k] = w[k] sum_m (x[m] w[m]) conj(w[k - m]),   w[j] = exp(-i pi j^2 / n),
// which follows from m k = (m^2 + k^2 - (k - m)^2) / 2: the sum is a linear
// convolution, done as a circular one of a 7-smooth length L >= 2n - 1 with
// the Stockham engine (forward, multiply by the precomputed transform of the
// conjugate chirp with 1/L folded in, inverse). The inverse DFT is the
// conjugate of the forward DFT of the conjugate. The chirp reduces j^2 modulo
// 2n in integers; both Bluestein tables are computed in FP64 on the host at
// plan creation and rounded once to FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <math.h>
#include <stdlib.h>

#include <vector>

#include "fft_reg.cuh"
#include "gfc_internal.h"

namespace gfc {
namespace {

constexpr int kExactThreads = 256;

template <typename T> __device__ __forceinline__ float ex_ld(const T* p);
template <> __device__ __forceinline__ float ex_ld<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ex_ld<__half>(const __half* p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float ex_ld<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <typename T> __device__ __forceinline__ T ex_st(float x);
template <> __device__ __forceinline__ float ex_st<float>(float x) { return x; }
template <> __device__ __forceinline__ __half ex_st<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 ex_st<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// ---- one DFT of length d.n on a shared-memory row ------------------------------------
struct DimArgs {
  int n, L;           // L = 0: n is 7-smooth (direct)
  FftPlan plan;       // schedule of n (direct) or L (Bluestein)
  const float2* tw;   // roots of unity of the scheduled length
  const float2* chirp;
  const float2* cf;
};

// DFT of the n values in b0 (DIR -1 forward, +1 unnormalised inverse); b0, b1
// are shared buffers of max(n, L) complex. Callers synchronise before; the
// result is visible to the whole block on return.
template <int DIR>
__device__ float2* dft_row(float2* b0, float2* b1, const DimArgs& d, int tid, int nthr) {
  // input is in b0[0..n); returns the buffer holding the n outputs
  if (d.L == 0) return fft_smem<DIR>(b0, b1, d.plan, 1, 1, d.tw, tid, nthr);
  // Bluestein: a[m] = x[m] w[m] (conj of the input for the inverse), zero to L
  for (int m = tid; m < d.L; m += nthr) {
    float2 v = make_float2(0.0f, 0.0f);
    if (m < d.n) {
      float2 x = b0[m];
      if (DIR > 0) x = cconj(x);
      v = cmul(x, __ldg(d.chirp + m));
    }
    b1[m] = v;
  }
  __syncthreads();
  float2* A = fft_smem<-1>(b1, b0, d.plan, 1, 1, d.tw, tid, nthr);
  float2* B = (A == b0) ? b1 : b0;
  for (int k = tid; k < d.L; k += nthr) A[k] = cmul(A[k], __ldg(d.cf + k));
  __syncthreads();
  float2* C = fft_smem<+1>(A, B, d.plan, 1, 1, d.tw, tid, nthr);
  for (int k = tid; k < d.n; k += nthr) {
    float2 y = cmul(C[k], __ldg(d.chirp + k));
    if (DIR > 0) y = cconj(y);
    C[k] = y;
  }
  __syncthreads();
  return C;
}

// rows of X (count rows of d.n complex, row stride ld) transformed in place
template <int DIR>
__global__ void __launch_bounds__(kExactThreads) k_exact_rows(float2* X, long long rows, int ld, DimArgs d) {
  extern __shared__ float2 sm[];
  const int len = d.L > d.n ? d.L : d.n;
  float2* b0 = sm;
  float2* b1 = sm + len;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    float2* x = X + r * ld;
    for (int m = threadIdx.x; m < d.n; m += blockDim.x) b0[m] = x[m];
    __syncthreads();
    float2* y = dft_row<DIR>(b0, b1, d, threadIdx.x, blockDim.x);
    for (int k = threadIdx.x; k < d.n; k += blockDim.x) x[k] = y[k];
    __syncthreads();
  }
}

// column l of a field (row l of the transposed array): forward DFT of length M,
// times G[k][min(l, N - l)] (G real and even, 1/(MN) folded in), inverse DFT
__global__ void __launch_bounds__(kExactThreads) k_exact_cols(float2* XT, int nf, int M, int N, int Nh,
                                                              const float* __restrict__ G, DimArgs d) {
  extern __shared__ float2 sm[];
  const int len = d.L > d.n ? d.L : d.n;
  float2* b0 = sm;
  float2* b1 = sm + len;
  const long long rows = (long long)nf * N;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int l = (int)(r % N);
    const int lg = l <= N - l ? l : N - l;
    float2* x = XT + r * M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) b0[m] = x[m];
    __syncthreads();
    float2* y = dft_row<-1>(b0, b1, d, threadIdx.x, blockDim.x);
    float2* z = (y == b0) ? b1 : b0;
    for (int k = threadIdx.x; k < M; k += blockDim.x) z[k] = cscale(y[k], __ldg(G + (size_t)k * Nh + lg));
    __syncthreads();
    float2* u = dft_row<+1>(z, y, d, threadIdx.x, blockDim.x);
    for (int k = threadIdx.x; k < M; k += blockDim.x) x[k] = u[k];
    __syncthreads();
  }
}

// ---- Bluestein rows with L = 2430 = 45 x 54, in registers ---------------------
// The same identity as dft_row on the register-resident schedule of the row
// passes: a block takes F = 2 rows of the pair tori at a time (persistent),
// T = 54 threads per row. Element m = t + 54 r of the chirp-multiplied row
// (zero past n) lands in thread t's registers; a length-45 DFT, one exchange,
// then threads j < 45 take the length-54 DFTs over r with twiddles w_L^(r j),
// giving A[j + 45 q]. Times the chirp filter's transform (1/L folded in), the
// spectrum goes back to shared memory in natural order, and the same two
// stages with conjugate twiddles give the unnormalised inverse; times the
// chirp, it replaces the row. Rows of length n with 2n - 1 <= 2430 whose
// Bluestein length is 2430 (n = 1202 .. 1215, e.g. 1208 for a 1200-wide image)
// take it; other lengths run the shared-memory engine.
struct ExRegRows {
  static constexpr int L = 2430, R1 = 45, R2 = 54, F = 2, T = R2;
  static constexpr int R1P = R1 + 2;  // odd R1: the exchange stride R1 + 2 spreads 8-byte words over the banks
  static constexpr int NP = (L / R1) * R1P;  // per-row exchange (also holds the spectrum in natural order)
  static constexpr int THREADS = ((F * T + 31) / 32) * 32;
  static_assert(R1 * R2 == L && R1 < R2 && NP >= L, "schedule");
  static constexpr size_t smem_bytes() { return (size_t)(R1 * R2 + F * NP) * sizeof(float2); }
};

template <int DIR>
__global__ void __launch_bounds__(ExRegRows::THREADS, 2) k_exact_rows_reg(float2* X, long long rows, int ld,
                                                                         DimArgs d) {
  using S = ExRegRows;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw2 = sm;                  // [R1][R2]: w_L^(r j)
  float2* buf = sm + S::R1 * S::R2;  // [F][NP]
  const int tid = threadIdx.x, f = tid / S::T, t = tid - f * S::T;
  const bool act = f < S::F, act2 = act && t < S::R1;
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    tw2[i] = d.tw[r * j];
  }
  float2* mybuf = buf + (act ? f : 0) * S::NP;
  const long long items = (rows + S::F - 1) / S::F;
  __syncthreads();
#pragma unroll 1
  for (long long w = blockIdx.x; w < items; w += gridDim.x) {
    const long long row = w * S::F + f;
    const bool vr = act && row < rows;
    float2* x = X + (vr ? row : 0) * (long long)ld;
    float2 v[S::R1];
#pragma unroll
    for (int r = 0; r < S::R1; ++r) {
      const int m = t + S::R2 * r;
      float2 a = make_float2(0.0f, 0.0f);
      if (vr && m < d.n) {
        float2 xm = x[m];
        if (DIR > 0) xm = cconj(xm);
        a = cmul(xm, __ldg(d.chirp + m));
      }
      v[r] = a;
    }
    if (act) {
      dft_reg<S::R1, -1>(v);
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();
    float2 u[S::R2];
    if (act2) {
      u[0] = mybuf[t];
#pragma unroll
      for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[t + S::R1P * r], tw2[t * S::R2 + r]);
      dft_reg<S::R2, -1>(u);
#pragma unroll
      for (int s2 = 0; s2 < S::R2; ++s2) u[s2] = cmul(u[s2], __ldg(d.cf + t + S::R1 * s2));
    }
    __syncthreads();  // the exchange read: it takes the spectrum in natural order
    if (act2) {
#pragma unroll
      for (int s2 = 0; s2 < S::R2; ++s2) mybuf[t + S::R1 * s2] = u[s2];
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int r = 0; r < S::R1; ++r) v[r] = mybuf[t + S::R2 * r];
      dft_reg<S::R1, +1>(v);
    }
    __syncthreads();  // the spectrum read: the exchange again
    if (act) {
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();
    if (act2) {
      u[0] = mybuf[t];
#pragma unroll
      for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[t + S::R1P * r], cconj(tw2[t * S::R2 + r]));
      dft_reg<S::R2, +1>(u);
#pragma unroll
      for (int s2 = 0; s2 < S::R2; ++s2) {
        const int k = t + S::R1 * s2;
        if (vr && k < d.n) {
          float2 y = cmul(u[s2], __ldg(d.chirp + k));
          if (DIR > 0) y = cconj(y);
          x[k] = y;
        }
      }
    }
    __syncthreads();  // the exchange free for the next rows
  }
}

// ---- the column direction by the recursive column solve --------------------
// After the row DFTs, column l of Eq. 23's Green multiply (G = 1/(M N lambda),
// lambda(k, l) = 2 cos(2 pi k / M) - b_l, b_l = 4 - 2 cos(2 pi l / N)) is, with
// the unnormalised inverse column DFT folded in, 1/N times the inverse of the
// cyclic tridiagonal operator S + S^-1 - b_l along the torus rows. With
// a + 1/a = b_l, a < 1, that inverse is -a / (1 - a^2) [(1 - a S)^-1 +
// (1 - a S^-1)^-1 - 1]: a causal and an anticausal first-order recursion
// around the cycle. It is real, so it maps the packed pair's real and
// imaginary parts each to its own solution, and it depends on l only through
// min(l, N - l). The rows are cut into segments of kExSeg (the last one
// shorter); each segment's recursions run in registers from zero carries,
// a sweep per column folds the segments' end values around the cycle into
// the carries, and each segment then solves with its carries.
// Per column (FP64, rounded once): 1 - a, a, C = -a / ((1 - a^2) N),
// 1 / (1 - a^M), a^kExSeg, a^(rows of the last segment); column 0 (b = 2,
// singular) is solved exactly (k_exact_col0).
constexpr int kExSeg = 16;

__global__ void k_exact_colcoef(float* cc, int M, int N, int Nh) {
  const int nseg = (M + kExSeg - 1) / kExSeg, last = M - kExSeg * (nseg - 1);
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < Nh; l += gridDim.x * blockDim.x) {
    float* c = cc + (size_t)l * 8;
    if (l == 0) {
      for (int i = 0; i < 8; ++i) c[i] = 0.0f;
      continue;
    }
    const double sn = sinpi((double)l / (double)N);
    const double d = 4.0 * sn * sn;  // b - 2
    const double r = sqrt(d * (4.0 + d));
    const double a = 2.0 / (2.0 + d + r), delta = (d + r) / (2.0 + d + r);
    c[0] = (float)delta;
    c[1] = (float)a;
    c[2] = (float)(-a / (delta * (1.0 + a) * (double)N));
    c[3] = (float)(1.0 / (1.0 - pow(a, (double)M)));
    c[4] = (float)pow(a, (double)kExSeg);
    c[5] = (float)pow(a, (double)last);
    c[6] = c[7] = 0.0f;
  }
}

// y <- x + a y as (x + y) - delta y (delta = 1 - a held to full precision)
__device__ __forceinline__ float2 ex_step(float2 x, float2 y, float delta) {
  return make_float2(__fmaf_rn(-delta, y.x, __fadd_rn(x.x, y.x)), __fmaf_rn(-delta, y.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 ex_fma(float T, float2 c, float2 e) {
  return make_float2(__fmaf_rn(T, c.x, e.x), __fmaf_rn(T, c.y, e.y));
}

// Scratch of pair torus q in the (otherwise unused) transpose buffer, complex
// elements from q M N: the segments' sums [nseg][2][N] (causal value at the
// segment's last row, anticausal value at its first row, from zero carries),
// then their carries [nseg][2][N] (into the segment from above, from below).
// 4 nseg N <= M N for every M >= 4.

// Segment sums, one lane per column l >= 1 (coalesced rows), the segment's
// rows in registers. Grid: (32-column strips / 4, segments, pairs).
__global__ void __launch_bounds__(128) k_exact_seg_sums(const float2* __restrict__ X, float2* __restrict__ XT, int M,
                                                        int N, int nseg, const float* __restrict__ cc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = (blockIdx.x * 4 + warp) * 32 + lane;
  if (l == 0 || l >= N) return;  // no lane waits on another
  const int lg = l <= N - l ? l : N - l;
  const float delta = __ldg(cc + (size_t)lg * 8);
  const int sg = blockIdx.y, r0 = sg * kExSeg, nr = min(kExSeg, M - r0);
  const float2* x = X + (size_t)blockIdx.z * M * N + (size_t)r0 * N + l;
  float2 v[kExSeg];
#pragma unroll
  for (int r = 0; r < kExSeg; ++r) v[r] = r < nr ? x[(size_t)r * N] : make_float2(0.0f, 0.0f);
  float2 e = make_float2(0.0f, 0.0f), ep = e;
#pragma unroll
  for (int r = 0; r < kExSeg; ++r)
    if (r < nr) e = ex_step(v[r], e, delta);
#pragma unroll
  for (int r = kExSeg - 1; r >= 0; --r)
    if (r < nr) ep = ex_step(v[r], ep, delta);
  float2* sums = XT + (size_t)blockIdx.z * M * N;
  sums[(size_t)(2 * sg) * N + l] = e;
  sums[(size_t)(2 * sg + 1) * N + l] = ep;
}

// The sweep, one thread per column l >= 1: the causal sums folded down the
// torus from a zero carry give y[M-1] = fold / (1 - a^M), which is the carry
// into segment 0 (row 0 follows row M-1); the carries follow segment by
// segment. The anticausal sums folded up give y'[0], the carry from below the
// last segment. Grid: (columns / 128, pairs).
__global__ void __launch_bounds__(128) k_exact_seg_sweep(float2* __restrict__ XT, int M, int N, int nseg,
                                                         const float* __restrict__ cc) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l == 0 || l >= N) return;
  const int lg = l <= N - l ? l : N - l;
  const float inv = __ldg(cc + (size_t)lg * 8 + 3), Ts = __ldg(cc + (size_t)lg * 8 + 4),
              Tl = __ldg(cc + (size_t)lg * 8 + 5);
  const float2* sums = XT + (size_t)blockIdx.y * M * N + l;
  float2* car = XT + (size_t)blockIdx.y * M * N + (size_t)2 * nseg * N + l;
  float2 t = make_float2(0.0f, 0.0f);
#pragma unroll 4
  for (int sg = 0; sg < nseg; ++sg) t = ex_fma(sg == nseg - 1 ? Tl : Ts, t, sums[(size_t)(2 * sg) * N]);
  float2 c = make_float2(t.x * inv, t.y * inv);  // y[M-1]: the carry into segment 0
#pragma unroll 4
  for (int sg = 0; sg < nseg; ++sg) {
    car[(size_t)(2 * sg) * N] = c;
    c = ex_fma(sg == nseg - 1 ? Tl : Ts, c, sums[(size_t)(2 * sg) * N]);
  }
  float2 q = make_float2(0.0f, 0.0f);
#pragma unroll 4
  for (int sg = nseg - 1; sg >= 0; --sg) q = ex_fma(sg == nseg - 1 ? Tl : Ts, q, sums[(size_t)(2 * sg + 1) * N]);
  c = make_float2(q.x * inv, q.y * inv);  // y'[0]: the carry from below the last segment
#pragma unroll 4
  for (int sg = nseg - 1; sg >= 0; --sg) {
    car[(size_t)(2 * sg + 1) * N] = c;
    c = ex_fma(sg == nseg - 1 ? Tl : Ts, c, sums[(size_t)(2 * sg + 1) * N]);
  }
}

// Each segment with its carries: the causal recursion down, the anticausal one
// up, U = C (y + y' - x) written over X. Grid as k_exact_seg_sums.
__global__ void __launch_bounds__(128) k_exact_seg_solve(float2* __restrict__ X, const float2* __restrict__ XT, int M,
                                                         int N, int nseg, const float* __restrict__ cc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = (blockIdx.x * 4 + warp) * 32 + lane;
  if (l == 0 || l >= N) return;
  const int lg = l <= N - l ? l : N - l;
  const float delta = __ldg(cc + (size_t)lg * 8), C = __ldg(cc + (size_t)lg * 8 + 2);
  const int sg = blockIdx.y, r0 = sg * kExSeg, nr = min(kExSeg, M - r0);
  float2* x = X + (size_t)blockIdx.z * M * N + (size_t)r0 * N + l;
  const float2* car = XT + (size_t)blockIdx.z * M * N + (size_t)2 * nseg * N + l;
  float2 v[kExSeg], y[kExSeg];
#pragma unroll
  for (int r = 0; r < kExSeg; ++r) v[r] = r < nr ? x[(size_t)r * N] : make_float2(0.0f, 0.0f);
  float2 yc = car[(size_t)(2 * sg) * N], ya = car[(size_t)(2 * sg + 1) * N];
#pragma unroll
  for (int r = 0; r < kExSeg; ++r) {
    yc = ex_step(v[r], yc, delta);
    y[r] = yc;
  }
#pragma unroll
  for (int r = kExSeg - 1; r >= 0; --r)
    if (r < nr) {
      ya = ex_step(v[r], ya, delta);
      x[(size_t)r * N] = make_float2(C * ((y[r].x + ya.x) - v[r].x), C * ((y[r].y + ya.y) - v[r].y));
    }
}

__device__ __forceinline__ double ex_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double ex_warp_exscan(double v) {
  const int lane = threadIdx.x & 31;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

// Column 0 of each pair torus (one warp each, FP64, the real and the imaginary
// part in turn): with d[r] = u[r+1] - u[r], (S + S^-1 - 2) u = f - mean(f)
// reads d[r] - d[r-1] = f[r] - mean(f); periodicity fixes d[-1] = -sum_r P[r] / M
// with P the prefix sums of f - mean(f); u[0] = 0 (a constant in column 0 is a
// constant in the field, which Algorithm B's offset removes). Each lane walks
// a contiguous run of rows; u / N replaces the column.
__global__ void __launch_bounds__(32) k_exact_col0(float2* __restrict__ X, int M, int N) {
  const int lane = threadIdx.x;
  float2* col = X + (size_t)blockIdx.x * M * N;
  const int run = (M + 31) / 32;
  const int r0 = min(lane * run, M), r1 = min(r0 + run, M);
  const double invM = 1.0 / (double)M, invN = 1.0 / (double)N;
  for (int part = 0; part < 2; ++part) {
    auto f = [&](int r) -> double { return part ? (double)col[(size_t)r * N].y : (double)col[(size_t)r * N].x; };
    double s0 = 0.0;
    for (int r = r0; r < r1; ++r) s0 += f(r);
    const double mean = ex_warp_sum(s0) * invM;
    const double off = ex_warp_exscan(s0 - mean * (double)(r1 - r0));
    double Pr = off, Ps = 0.0;
    for (int r = r0; r < r1; ++r) {
      Pr += f(r) - mean;
      Ps += Pr;
    }
    const double D = -ex_warp_sum(Ps) * invM;
    double u = ex_warp_exscan(D * (double)(r1 - r0) + Ps);
    Pr = off;
    for (int r = r0; r < r1; ++r) {
      const double fr = f(r);  // read before the row is overwritten
      float2* cr = col + (size_t)r * N;
      if (part) cr->y = (float)(u * invN);
      else cr->x = (float)(u * invN);
      Pr += fr - mean;
      u += D + Pr;
    }
  }
}

// [R][Cn] -> [Cn][R] per field, 32 x 32 tiles through shared memory
__global__ void k_exact_transpose(const float2* __restrict__ src, float2* __restrict__ dst, int R, int Cn) {
  __shared__ float2 tile[32][33];
  const size_t fo = (size_t)blockIdx.z * R * Cn;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cn) tile[i][threadIdx.x] = src[fo + (size_t)r * Cn + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < Cn) dst[fo + (size_t)c * R + r] = tile[threadIdx.x][i];
  }
}

// L of field f at torus cell (r, c): image block at (p, p); MODE 0: L = div E
// (Eq. 3) of the (optionally edited) gradient, MODE 1: L given, MODE 2 (the
// adjoint): z = Crop^T(grad_out) - (sum grad_out) e_00, the sum from `gsum`
template <typename T, int MODE, int EDIT>
__device__ __forceinline__ float exact_lap(const T* __restrict__ in0, const T* __restrict__ in1, int f, int r, int c,
                                           int H, int W, int p, const EditArgs& ed, const double* __restrict__ gsum) {
  if (MODE == 2 && r == 0 && c == 0) return (float)(-gsum[f]);  // the image block starts at (p, p), p >= 1
  const int i = r - p, j = c - p;
  const int nrows = (MODE == 0) ? H + 1 : H, ncols = (MODE == 0) ? W + 1 : W;
  if (i < 0 || i >= nrows || j < 0 || j >= ncols) return 0.0f;
  const size_t fe = (size_t)H * W;
  const T* a = in0 + f * fe;
  if (MODE != 0) return ex_ld(a + (size_t)i * W + j);
  const T* b = in1 + f * fe;
  const T* e = (EDIT == kEditMerge) ? static_cast<const T*>(ed.edges) + f * fe : nullptr;
  const float t2 = (EDIT == kEditThreshold) ? ed.t2[f] : 0.0f;
  const float2 c0 = edit_pixel<T, EDIT>(a, b, e, i, j, H, W, t2, ed.alpha);
  return (c0.x - edit_pixel<T, EDIT>(a, b, e, i, j - 1, H, W, t2, ed.alpha).x) +
         (c0.y - edit_pixel<T, EDIT>(a, b, e, i - 1, j, H, W, t2, ed.alpha).y);
}

// Two fields per complex torus: X[q] = L[2q] + i L[2q + 1] (the second 0 when
// nf is odd). G is real and even, so the convolution maps the real and the
// imaginary part each to its own real solution.
template <typename T, int MODE, int EDIT>
__global__ void k_exact_load(const T* __restrict__ in0, const T* __restrict__ in1, float2* __restrict__ X, int nf,
                             int H, int W, int M, int N, int p, EditArgs ed, const double* __restrict__ gsum) {
  const int q = blockIdx.y, f0 = 2 * q, f1 = f0 + 1;
  float2* x = X + (size_t)q * M * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)M * N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / N), c = (int)(idx - (long long)r * N);
    const float v0 = exact_lap<T, MODE, EDIT>(in0, in1, f0, r, c, H, W, p, ed, gsum);
    const float v1 = f1 < nf ? exact_lap<T, MODE, EDIT>(in0, in1, f1, r, c, H, W, p, ed, gsum) : 0.0f;
    x[idx] = make_float2(v0, v1);
  }
}

// adjoint: the sum of each field's grad_out, one block per field; each thread
// adds its elements in FP32 in runs of 16, then in FP64; the block combines the
// threads in a fixed order
constexpr int kSumThreads = 1024;
template <typename T>
__global__ void __launch_bounds__(kSumThreads) k_exact_gsum(const T* __restrict__ g, int H, int W,
                                                           double* __restrict__ gsum) {
  const size_t fe = (size_t)H * W;
  const T* a = g + (size_t)blockIdx.x * fe;
  double acc = 0.0;
  float run = 0.0f;
  int k = 0;
  for (size_t i = threadIdx.x; i < fe; i += kSumThreads) {
    run += ex_ld(a + i);
    if (++k == 16) {
      acc += (double)run;
      run = 0.0f;
      k = 0;
    }
  }
  acc += (double)run;
  __shared__ double red[kSumThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) s += red[w];
    gsum[blockIdx.x] = s;
  }
}

// out[i][j] = u[p + i][p + j] - u[0][0] (Algorithm B), u the real (even field)
// or imaginary (odd field) part of the pair's solution
template <typename T>
__global__ void k_exact_out(const float2* __restrict__ X, T* __restrict__ out, int H, int W, int M, int N, int p) {
  const int f = blockIdx.y;
  const float* x = reinterpret_cast<const float*>(X + (size_t)(f / 2) * M * N) + (f & 1);
  const float u00 = x[0];
  T* o = out + (size_t)f * H * W;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)H * W;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / W), j = (int)(idx - (long long)i * W);
    o[idx] = ex_st<T>(x[2 * ((size_t)(p + i) * N + (p + j))] - u00);
  }
}

// adjoint: grad_gx[i][j] = w[p+i][p+j] - w[p+i][p+j+1], grad_gy[i][j] =
// w[p+i][p+j] - w[p+i+1][p+j] (the transpose of the divergence), w the real
// (even field) or imaginary (odd field) part of the pair's convolution
template <typename T>
__global__ void k_exact_out_adj(const float2* __restrict__ X, T* __restrict__ ggx, T* __restrict__ ggy, int H, int W,
                                int M, int N, int p) {
  const int f = blockIdx.y;
  const float* x = reinterpret_cast<const float*>(X + (size_t)(f / 2) * M * N) + (f & 1);
  T* ox = ggx + (size_t)f * H * W;
  T* oy = ggy + (size_t)f * H * W;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)H * W;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / W), j = (int)(idx - (long long)i * W);
    const size_t at = (size_t)(p + i) * N + (p + j);  // p + W < N, p + H < M
    const float w0 = x[2 * at];
    ox[idx] = ex_st<T>(w0 - x[2 * (at + 1)]);
    oy[idx] = ex_st<T>(w0 - x[2 * (at + N)]);
  }
}

int smooth_at_least(int x) {
  int n = x;
  while (!is_7smooth(n)) ++n;
  return n;
}

DimArgs dim_args(const ExactDim& d) {
  DimArgs a;
  a.n = d.n;
  a.L = d.L;
  a.plan = d.plan;
  a.tw = d.tw;
  a.chirp = d.chirp;
  a.cf = d.cf;
  return a;
}

size_t dim_smem(const ExactDim& d) { return 2 * (size_t)(d.L > d.n ? d.L : d.n) * sizeof(float2); }

template <typename K>
cudaError_t raise_smem(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Bluestein tables in FP64 on the host, rounded once to FP32:
//   chirp[j] = exp(-i pi (j^2 mod 2n) / n),                       j < n
//   cf[k]    = (1/L) sum_j c[j] exp(-2 pi i (j k mod L) / L),     k < L
// with c[j] = conj(chirp[|j|]) for |j| < n placed circularly (c[L - j] = c[j]).
// The O(L n) sum uses a table of the L-th roots indexed by exact integer
// reduction; plan creation only.
static std::vector<float2> host_chirp(int n) {
  std::vector<float2> w(n);
  for (int j = 0; j < n; ++j) {
    const long long q = ((long long)j * j) % (2LL * n);
    const double a = M_PI * (double)q / (double)n;
    w[j] = make_float2((float)cos(a), (float)-sin(a));
  }
  return w;
}

static std::vector<float2> host_bluestein(int n, int L) {
  std::vector<double> rc(L), rs(L);
  for (int r = 0; r < L; ++r) {
    const double a = 2.0 * M_PI * (double)r / (double)L;
    rc[r] = cos(a);
    rs[r] = -sin(a);  // exp(-2 pi i r / L)
  }
  std::vector<double> re(L, 0.0), im(L, 0.0);
  for (int j = -(n - 1); j <= n - 1; ++j) {
    const long long aj = j < 0 ? -j : j;
    const long long q = (aj * aj) % (2LL * n);
    const double a = M_PI * (double)q / (double)n;
    const double cr = cos(a), ci = sin(a);  // conj(chirp[|j|]) = exp(+i pi q / n)
    const int jj = j < 0 ? j + L : j;
    int idx = 0;
    for (int k = 0; k < L; ++k) {
      re[k] += cr * rc[idx] - ci * rs[idx];
      im[k] += cr * rs[idx] + ci * rc[idx];
      idx += jj;
      if (idx >= L) idx -= L;
    }
  }
  std::vector<float2> cf(L);
  for (int k = 0; k < L; ++k) cf[k] = make_float2((float)(re[k] / L), (float)(im[k] / L));
  return cf;
}

cudaError_t setup_dim(ExactDim* d, int n, cudaStream_t s) {
  d->n = n;
  d->L = is_7smooth(n) ? 0 : smooth_at_least(2 * n - 1);
  const int len = d->L ? d->L : n;
  if (!make_fft_plan(len, &d->plan)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMalloc(&d->tw, (size_t)len * sizeof(float2));
  if (e == cudaSuccess) e = build_twiddles(d->tw, len, s);
  if (e == cudaSuccess && d->L) {
    const std::vector<float2> w = host_chirp(n), cf = host_bluestein(n, d->L);
    e = cudaMalloc(&d->chirp, (size_t)n * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&d->cf, (size_t)d->L * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(d->chirp, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->cf, cf.data(), cf.size() * sizeof(float2), cudaMemcpyHostToDevice);
  }
  return e;
}

template <typename T, int MODE>
cudaError_t run_exact(gfc_plan* P, const Bufs& bf, const T* in0, const T* in1, T* out0, T* out1, int nf,
                      cudaStream_t st, const EditArgs* ed) {
  const int M = P->M, N = P->N;
  const int np = (nf + 1) / 2;  // complex tori: two fields each
  float2* X = bf.spec;
  float2* XT = bf.spec + (size_t)np * M * N;
  const EditArgs none{kEditNone, 0.0f, nullptr, nullptr, nullptr, nullptr};
  const EditArgs& E = ed ? *ed : none;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const DimArgs dr = dim_args(P->ex_row), dc = dim_args(P->ex_col);
  const size_t sr = dim_smem(P->ex_row), sc = dim_smem(P->ex_col);
  cudaError_t e;
  double* gsum = reinterpret_cast<double*>(bf.partial);  // MODE 2: sum(grad_out) per field
  if (MODE == 2) {
    prof_begin(P, 3, st);
    k_exact_gsum<T><<<nf, kSumThreads, 0, st>>>(in0, P->H, P->W, gsum);
    prof_end(P, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // divergence / Laplacian / Crop^T(grad_out) into the complex tori
  {
    const long long cells = (long long)M * N;
    int gx = (int)((cells + kExactThreads - 1) / kExactThreads);
    if (gx > 4 * sms) gx = 4 * sms;
    const dim3 g(gx, np);
    const int H = P->H, W = P->W, p = P->pad;
    if (MODE == 2)
      k_exact_load<T, 2, kEditNone><<<g, kExactThreads, 0, st>>>(in0, in1, X, nf, H, W, M, N, p, E, gsum);
    else if (MODE == 1)
      k_exact_load<T, 1, kEditNone><<<g, kExactThreads, 0, st>>>(in0, in1, X, nf, H, W, M, N, p, E, gsum);
    else if (E.kind == kEditThreshold)
      k_exact_load<T, 0, kEditThreshold><<<g, kExactThreads, 0, st>>>(in0, in1, X, nf, H, W, M, N, p, E, gsum);
    else if (E.kind == kEditMerge)
      k_exact_load<T, 0, kEditMerge><<<g, kExactThreads, 0, st>>>(in0, in1, X, nf, H, W, M, N, p, E, gsum);
    else
      k_exact_load<T, 0, kEditNone><<<g, kExactThreads, 0, st>>>(in0, in1, X, nf, H, W, M, N, p, E, gsum);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const long long rows = (long long)np * M;
  const int grow = (int)(rows < 8LL * sms ? rows : 8LL * sms);
  if ((e = raise_smem(k_exact_rows<-1>, sr)) != cudaSuccess) return e;
  if ((e = raise_smem(k_exact_rows<+1>, sr)) != cudaSuccess) return e;
  if ((e = raise_smem(k_exact_cols, sc)) != cudaSuccess) return e;
  // rows whose Bluestein length is the register schedule's run on it
  const bool reg_rows = P->ex_row.L == ExRegRows::L && getenv("GFC_EXACT_GENERIC_ROWS") == nullptr;
  const int greg = (int)(((rows + ExRegRows::F - 1) / ExRegRows::F) < 2LL * sms ? (rows + ExRegRows::F - 1) / ExRegRows::F
                                                                                 : 2LL * sms);
  if (reg_rows) {
    if ((e = raise_smem(k_exact_rows_reg<-1>, ExRegRows::smem_bytes())) != cudaSuccess) return e;
    if ((e = raise_smem(k_exact_rows_reg<+1>, ExRegRows::smem_bytes())) != cudaSuccess) return e;
  }
  prof_begin(P, 0, st);
  if (reg_rows)
    k_exact_rows_reg<-1><<<greg, ExRegRows::THREADS, ExRegRows::smem_bytes(), st>>>(X, rows, N, dr);
  else
    k_exact_rows<-1><<<grow, kExactThreads, sr, st>>>(X, rows, N, dr);
  prof_end(P, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (getenv("GFC_EXACT_COLUMN_DFT") == nullptr) {
    // the column direction by the recursive column solve, in place on the
    // row-major tori (XT holds the causal pass); column 0 exactly
    prof_begin(P, 1, st);
    const int strips = (N + 31) / 32, nseg = (M + kExSeg - 1) / kExSeg;
    const dim3 sgrid((strips + 3) / 4, nseg, np);
    k_exact_seg_sums<<<sgrid, 128, 0, st>>>(X, XT, M, N, nseg, P->colcoef);
    k_exact_seg_sweep<<<dim3((N + 127) / 128, np), 128, 0, st>>>(XT, M, N, nseg, P->colcoef);
    k_exact_seg_solve<<<sgrid, 128, 0, st>>>(X, XT, M, N, nseg, P->colcoef);
    k_exact_col0<<<np, 32, 0, st>>>(X, M, N);
    P->prof.launches[1] += 3;  // four launches in this pass
    prof_end(P, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    // the column DFTs (Bluestein where M is not 7-smooth) on the transposed tori
    const dim3 tb(32, 8);
    k_exact_transpose<<<dim3((N + 31) / 32, (M + 31) / 32, np), tb, 0, st>>>(X, XT, M, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long cols = (long long)np * N;
    prof_begin(P, 1, st);
    k_exact_cols<<<(int)(cols < 8LL * sms ? cols : 8LL * sms), kExactThreads, sc, st>>>(XT, np, M, N, P->Nh, P->G,
                                                                                         dc);
    prof_end(P, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_exact_transpose<<<dim3((M + 31) / 32, (N + 31) / 32, np), tb, 0, st>>>(XT, X, N, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  prof_begin(P, 2, st);
  if (reg_rows)
    k_exact_rows_reg<+1><<<greg, ExRegRows::THREADS, ExRegRows::smem_bytes(), st>>>(X, rows, N, dr);
  else
    k_exact_rows<+1><<<grow, kExactThreads, sr, st>>>(X, rows, N, dr);
  prof_end(P, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    const long long cells = (long long)P->H * P->W;
    int gx = (int)((cells + kExactThreads - 1) / kExactThreads);
    if (gx > 4 * sms) gx = 4 * sms;
    if (MODE == 2)
      k_exact_out_adj<T><<<dim3(gx, nf), kExactThreads, 0, st>>>(X, out0, out1, P->H, P->W, M, N, P->pad);
    else
      k_exact_out<T><<<dim3(gx, nf), kExactThreads, 0, st>>>(X, out0, P->H, P->W, M, N, P->pad);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t exact_setup(gfc_plan* P, cudaStream_t s) {
  cudaError_t e = setup_dim(&P->ex_row, P->N, s);
  if (e == cudaSuccess) e = setup_dim(&P->ex_col, P->M, s);
  // the recursive column solve's coefficients, [Nh] x 8 floats (freed with the plan)
  if (e == cudaSuccess && !P->colcoef) e = cudaMalloc(&P->colcoef, (size_t)P->Nh * 8 * sizeof(float));
  if (e == cudaSuccess) {
    k_exact_colcoef<<<(P->Nh + 255) / 256, 256, 0, s>>>(P->colcoef, P->M, P->N, P->Nh);
    e = cudaGetLastError();
  }
  return e;
}

void exact_release(gfc_plan* P) {
  for (ExactDim* d : {&P->ex_row, &P->ex_col}) {
    cudaFree(d->tw);
    cudaFree(d->chirp);
    cudaFree(d->cf);
    d->tw = d->chirp = d->cf = nullptr;
  }
}

cudaError_t run_chunk_exact(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                            void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  if (mode < 0 || mode > 2) return cudaErrorNotSupported;
  auto go = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    const T* a = static_cast<const T*>(in0);
    const T* b = static_cast<const T*>(in1);
    T* o = static_cast<T*>(out0);
    T* o1 = static_cast<T*>(out1);
    if (mode == 0) return run_exact<T, 0>(P, bf, a, b, o, o1, nf, st, ed);
    if (mode == 1) return run_exact<T, 1>(P, bf, a, b, o, o1, nf, st, ed);
    return run_exact<T, 2>(P, bf, a, b, o, o1, nf, st, ed);
  };
  switch (P->dtype) {
    case GFC_F32: return go(float{});
    case GFC_F16: return go(__half{});
    default: return go(__nv_bfloat16{});
  }
}

}  // namespace gfc

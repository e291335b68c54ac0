// edit.cu -- gradient-domain editing steps around the solve (Sec. 2.3.2, Sec. 3.2).
//
//  * per-field mean / standard deviation and the colour correction of Eq. 25;
//  * gradient thresholding at a fraction of the largest (or a given) magnitude
//    (Sec. 3.1.4, Sec. 3.2.3);
//  * gradient-domain merging, Eq. 26: |Ep| = |E|^(1-alpha) C^alpha, orientation kept;
//  * the boundary-preserving offset of Sec. 2.3.2 (least-squares constant over
//    a ring of padding, then the ring cropped).
//
// All of these are HBM-bound streams over [fields][H][W]. Fields whose size is
// a multiple of 4 elements are read and written in packs of 4 (16-byte FP32 or
// 8-byte 16-bit accesses); others element by element. A field is split into a
// fixed number of contiguous block ranges that depends only on its size, so
// every reduction runs in the same order on every call (deterministic). Sums
// are taken in FP32 over 16 elements per thread and accumulated in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <initializer_list>

#include "gfc_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerBlock = 16384;  // target elements per block
constexpr int kMaxBlocks = 256;   // per field: partials use half of the field's scratch
constexpr int kCoefOff = 1024;    // float offset of the per-field coefficients in its scratch
constexpr int kUnroll = 4;        // packs per thread per iteration

int blocks_for(long long n) {
  long long b = (n + kPerBlock - 1) / kPerBlock;
  return (int)(b < 1 ? 1 : (b > kMaxBlocks ? kMaxBlocks : b));
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T> __device__ __forceinline__ T from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_f<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// K consecutive elements (pack i) of a T array, as floats
template <typename T, int K> struct Pack {
  static __device__ __forceinline__ void ld(const T* p, long long i, float* v) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = to_f(p[i * K + k]);
  }
  static __device__ __forceinline__ void st(T* p, long long i, const float* v) {
#pragma unroll
    for (int k = 0; k < K; ++k) p[i * K + k] = from_f<T>(v[k]);
  }
  // copy with the stored bits where keep[k], 0 elsewhere
  static __device__ __forceinline__ void cp(const T* s, T* d, long long i, const bool* keep) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[i * K + k] = keep[k] ? s[i * K + k] : from_f<T>(0.0f);
  }
};
template <> struct Pack<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, long long i, float* v) {
    const float4 q = reinterpret_cast<const float4*>(p)[i];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  static __device__ __forceinline__ void st(float* p, long long i, const float* v) {
    reinterpret_cast<float4*>(p)[i] = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void cp(const float* s, float* d, long long i, const bool* keep) {
    float v[4];
    ld(s, i, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = keep[k] ? v[k] : 0.0f;
    st(d, i, v);
  }
};
template <typename T> struct Pack16x4 {
  static __device__ __forceinline__ void ld(const T* p, long long i, float* v) {
    const uint2 u = reinterpret_cast<const uint2*>(p)[i];
    const T* h = reinterpret_cast<const T*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = to_f(h[k]);
  }
  static __device__ __forceinline__ void st(T* p, long long i, const float* v) {
    uint2 u;
    T* h = reinterpret_cast<T*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = from_f<T>(v[k]);
    reinterpret_cast<uint2*>(p)[i] = u;
  }
  static __device__ __forceinline__ void cp(const T* s, T* d, long long i, const bool* keep) {
    uint2 u = reinterpret_cast<const uint2*>(s)[i];
    T* h = reinterpret_cast<T*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (!keep[k]) h[k] = from_f<T>(0.0f);
    reinterpret_cast<uint2*>(d)[i] = u;
  }
};
template <> struct Pack<__half, 4> : Pack16x4<__half> {};
template <> struct Pack<__nv_bfloat16, 4> : Pack16x4<__nv_bfloat16> {};

// block range [lo, hi) of pack indices handled by block b of nblk
__device__ __forceinline__ void block_range(long long n, int nblk, int b, long long* lo, long long* hi) {
  const long long per = (n + nblk - 1) / nblk;
  *lo = per * b;
  long long h = *lo + per;
  *hi = h < n ? h : n;
}

// sum of two doubles over the block, fixed order; result valid in thread 0
__device__ __forceinline__ double2 block_sum2(double a, double b) {
  __shared__ double2 red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = make_double2(a, b);
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) {
      r.x += red[i].x;
      r.y += red[i].y;
    }
  return r;
}

__device__ __forceinline__ float block_max(float m) {
  __shared__ float red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) r = fmaxf(r, red[i]);
  return r;
}

// ---- first and second moments -------------------------------------------------
// partial[f][b] = (sum d, sum d^2) with d = x - x[f][0] over block b's range
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_moments_partial(const T* __restrict__ a, long long n, int nblk,
                                                             float* __restrict__ scratch, int f0) {
  const int f = blockIdx.y, b = blockIdx.x;
  const T* x = a + (long long)(f0 + f) * n;
  const float shift = to_f(x[0]);
  long long lo, hi;
  block_range(n / K, nblk, b, &lo, &hi);
  double S = 0.0, Q = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += (long long)kUnroll * kThreads) {
    float v[kUnroll][K];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long j = i + (long long)u * kThreads;
      if (j < hi) {
        Pack<T, K>::ld(x, j, v[u]);
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[u][k] = shift;
      }
    }
    float s = 0.f, q = 0.f;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float d = v[u][k] - shift;
        s += d;
        q = fmaf(d, d, q);
      }
    S += s;
    Q += q;
  }
  const double2 r = block_sum2(S, Q);
  if (threadIdx.x == 0) reinterpret_cast<double2*>(scratch + (size_t)f * gfc::kMaxRowBlocks)[b] = r;
}

// One warp per field: combine the block partials in a fixed order into
// (mean, std) at kCoefOff of the field's scratch; also to the caller's arrays.
template <typename T>
__global__ void k_moments_finish(const T* __restrict__ a, long long n, int nblk, float* __restrict__ scratch,
                                 int f0, int nf, float* __restrict__ mean_out, float* __restrict__ std_out) {
  const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (f >= nf) return;
  float* sc = scratch + (size_t)f * gfc::kMaxRowBlocks;
  const double2* part = reinterpret_cast<const double2*>(sc);
  double S = 0.0, Q = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    S += part[b].x;
    Q += part[b].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S += __shfl_down_sync(0xffffffffu, S, o);
    Q += __shfl_down_sync(0xffffffffu, Q, o);
  }
  if (lane == 0) {
    const double shift = (double)to_f(a[(long long)(f0 + f) * n]);
    const double md = S / (double)n;
    double var = Q / (double)n - md * md;
    if (var < 0.0) var = 0.0;
    const float mean = (float)(shift + md), sd = (float)sqrt(var);
    sc[kCoefOff] = mean;
    sc[kCoefOff + 1] = sd;
    if (mean_out) mean_out[f0 + f] = mean;
    if (std_out) std_out[f0 + f] = sd;
  }
}

// Eq. 25 in place: x <- (x - mean_c) * ref_std / std_c + ref_mean
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_color_apply(T* __restrict__ a, long long n, int nblk,
                                                         const float* __restrict__ scratch, int f0,
                                                         const float* __restrict__ ref_mean,
                                                         const float* __restrict__ ref_std) {
  const int f = blockIdx.y, b = blockIdx.x;
  const float* sc = scratch + (size_t)f * gfc::kMaxRowBlocks + kCoefOff;
  const float mc = sc[0], sdc = sc[1];
  const float mi = ref_mean[f0 + f], si = ref_std[f0 + f];
  const float g = sdc > 0.f ? si / sdc : 0.f;
  T* x = a + (long long)(f0 + f) * n;
  long long lo, hi;
  block_range(n / K, nblk, b, &lo, &hi);
  for (long long i = lo + threadIdx.x; i < hi; i += (long long)kUnroll * kThreads) {
    float v[kUnroll][K];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long j = i + (long long)u * kThreads;
      if (j < hi) Pack<T, K>::ld(x, j, v[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long j = i + (long long)u * kThreads;
      if (j < hi) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[u][k] = fmaf(v[u][k] - mc, g, mi);
        Pack<T, K>::st(x, j, v[u]);
      }
    }
  }
}

// ---- gradient thresholding ------------------------------------------------------
using gfc::edit_mag2;

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_mag_max_partial(const T* __restrict__ gx, const T* __restrict__ gy,
                                                             long long n, int nblk, float* __restrict__ scratch,
                                                             int f0) {
  const int f = blockIdx.y, b = blockIdx.x;
  const T* x = gx + (long long)(f0 + f) * n;
  const T* y = gy + (long long)(f0 + f) * n;
  long long lo, hi;
  block_range(n / K, nblk, b, &lo, &hi);
  float m = 0.f;
  for (long long i = lo + threadIdx.x; i < hi; i += (long long)kUnroll * kThreads) {
    float vx[kUnroll][K], vy[kUnroll][K];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long j = i + (long long)u * kThreads;
      if (j < hi) {
        Pack<T, K>::ld(x, j, vx[u]);
        Pack<T, K>::ld(y, j, vy[u]);
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) vx[u][k] = vy[u][k] = 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < K; ++k) m = fmaxf(m, edit_mag2(vx[u][k], vy[u][k]));
  }
  m = block_max(m);
  if (threadIdx.x == 0) scratch[(size_t)f * gfc::kMaxRowBlocks + b] = m;
}

// One warp per field: t2[f] = fl(t * t), t = fl(frac * r), with r = ref when
// ref > 0, else r = fl(sqrt(max m2)) over the field's partial maxima.
__global__ void k_threshold_finish(const float* __restrict__ scratch, int nblk, int f0, int nf, float frac,
                                   float ref, float* __restrict__ t2) {
  const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (f >= nf) return;
  float r = ref;
  if (!(ref > 0.f)) {
    float m = 0.f;
    const float* part = scratch + (size_t)f * gfc::kMaxRowBlocks;
    for (int i = lane; i < nblk; i += 32) m = fmaxf(m, part[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    r = __fsqrt_rn(m);
  }
  const float t = __fmul_rn(frac, r);
  if (lane == 0) t2[f0 + f] = __fmul_rn(t, t);
}

// kept values are copied with their stored bits; outputs may be the inputs
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_threshold_apply(const T* gx, const T* gy, long long n, int nblk,
                                                             const float* __restrict__ t2s, int f0, T* ox, T* oy) {
  const int f = blockIdx.y, b = blockIdx.x;
  const float t2 = t2s[f0 + f];
  const long long base = (long long)(f0 + f) * n;
  long long lo, hi;
  block_range(n / K, nblk, b, &lo, &hi);
  for (long long i = lo + threadIdx.x; i < hi; i += (long long)kUnroll * kThreads) {
    float vx[kUnroll][K], vy[kUnroll][K];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long j = i + (long long)u * kThreads;
      if (j < hi) {
        Pack<T, K>::ld(gx + base, j, vx[u]);
        Pack<T, K>::ld(gy + base, j, vy[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long j = i + (long long)u * kThreads;
      if (j < hi) {
        bool keep[K];
#pragma unroll
        for (int k = 0; k < K; ++k) keep[k] = !(edit_mag2(vx[u][k], vy[u][k]) < t2);
        Pack<T, K>::cp(gx + base, ox + base, j, keep);
        Pack<T, K>::cp(gy + base, oy + base, j, keep);
      }
    }
  }
}

// ---- gradient-domain merging, Eq. 26 ------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_merge(const T* gx, const T* gy, const T* __restrict__ edges,
                                                   long long packs, float alpha, T* ox, T* oy) {
  const long long stride = (long long)gridDim.x * kThreads;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < packs; i += stride) {
    float x[K], y[K], c[K];
    Pack<T, K>::ld(gx, i, x);
    Pack<T, K>::ld(gy, i, y);
    Pack<T, K>::ld(edges, i, c);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float s = gfc::edit_merge_scale(x[k], y[k], c[k], alpha);
      x[k] = __fmul_rn(x[k], s);
      y[k] = __fmul_rn(y[k], s);
    }
    Pack<T, K>::st(ox, i, x);
    Pack<T, K>::st(oy, i, y);
  }
}

// ---- boundary-preserving offset (Sec. 2.3.2) --------------------------------------
// ring pixel q of an H x W field: top rows, bottom rows, then the two side bands
__device__ __forceinline__ long long ring_index(long long q, int H, int W, int ring) {
  const long long band = (long long)ring * W;
  if (q < band) return q;
  if (q < 2 * band) return (long long)(H - ring) * W + (q - band);
  const long long s = q - 2 * band;
  const int r = ring + (int)(s / (2 * ring));
  const int k = (int)(s % (2 * ring));
  const int c = k < ring ? k : W - 2 * ring + k;
  return (long long)r * W + c;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ring_partial(const T* __restrict__ u, int H, int W, int ring,
                                                          long long nr, int nblk, float* __restrict__ scratch,
                                                          int f0) {
  const int f = blockIdx.y, b = blockIdx.x;
  const T* x = u + (long long)(f0 + f) * H * W;
  long long lo, hi;
  block_range(nr, nblk, b, &lo, &hi);
  double S = 0.0;
  for (long long q = lo + threadIdx.x; q < hi; q += kThreads) S += (double)to_f(x[ring_index(q, H, W, ring)]);
  const double2 r = block_sum2(S, 0.0);
  if (threadIdx.x == 0) reinterpret_cast<double*>(scratch + (size_t)f * gfc::kMaxRowBlocks)[b] = r.x;
}

// block b of a field writes inner rows [b rpb, (b + 1) rpb)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ring_apply(const T* __restrict__ u, int H, int W, int ring,
                                                        long long nr, int nblk_ring, int rpb,
                                                        const float* __restrict__ scratch, int f0,
                                                        T* __restrict__ inner) {
  const int f = blockIdx.y, b = blockIdx.x;
  __shared__ float s_c;
  if (threadIdx.x < 32) {
    const double* part = reinterpret_cast<const double*>(scratch + (size_t)f * gfc::kMaxRowBlocks);
    double S = 0.0;
    for (int i = threadIdx.x; i < nblk_ring; i += 32) S += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_down_sync(0xffffffffu, S, o);
    if (threadIdx.x == 0) s_c = (float)(S / (double)nr);
  }
  __syncthreads();
  const float c = s_c;
  const int Hi = H - 2 * ring, Wi = W - 2 * ring;
  const T* x = u + (long long)(f0 + f) * H * W;
  T* o = inner + (long long)(f0 + f) * Hi * Wi;
  const int r1 = min(Hi, (b + 1) * rpb);
  for (int i = b * rpb; i < r1; ++i) {
    const T* src = x + (long long)(i + ring) * W + ring;
    T* dst = o + (long long)i * Wi;
    for (int j = threadIdx.x; j < Wi; j += kThreads) dst[j] = from_f<T>(to_f(src[j]) - c);
  }
}

// ---- host side ---------------------------------------------------------------------
gfc_status check_uniform(gfc_plan* P, const char* fn) {
  if (!P) return gfc::fail(GFC_ERR_INVALID_ARG, "%s: null plan", fn);
  if (P->ragged) return gfc::fail(GFC_ERR_UNSUPPORTED, "%s: ragged plans are not supported", fn);
  if ((long long)P->H * P->W >= (1ll << 31))
    return gfc::fail(GFC_ERR_UNSUPPORTED, "%s: fields of 2^31 elements or more are not supported", fn);
  return GFC_OK;
}

int fields_of(const gfc_plan* P) { return P->batch * P->C; }
// fields per launch: the scratch holds one chunk of fields; grid.y <= 65535
int launch_fields(const gfc_plan* P) { return P->chunk < 65535 ? P->chunk : 65535; }

// packs of 4 when every field starts on a pack boundary and every pointer is aligned to one
bool packed4(const gfc_plan* P, std::initializer_list<const void*> ptrs) {
  const size_t pack = 4 * gfc::dtype_size(P->dtype);
  if (((long long)P->H * P->W) % 4 != 0) return false;
  for (const void* p : ptrs)
    if (reinterpret_cast<uintptr_t>(p) % pack != 0) return false;
  return true;
}

template <typename T>
gfc_status run_moments(gfc_plan* P, const void* a, float* mean_out, float* std_out) {
  const long long n = (long long)P->H * P->W;
  const int nblk = blocks_for(n), F = fields_of(P), L = launch_fields(P);
  const bool v4 = packed4(P, {a});
  float* sc = P->partial;
  for (int f0 = 0; f0 < F; f0 += L) {
    const int nf = F - f0 < L ? F - f0 : L;
    const dim3 g(nblk, nf);
    if (v4) k_moments_partial<T, 4><<<g, kThreads, 0, P->stream>>>((const T*)a, n, nblk, sc, f0);
    else k_moments_partial<T, 1><<<g, kThreads, 0, P->stream>>>((const T*)a, n, nblk, sc, f0);
    k_moments_finish<T><<<(nf + 7) / 8, 256, 0, P->stream>>>((const T*)a, n, nblk, sc, f0, nf, mean_out, std_out);
  }
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

template <typename T>
gfc_status run_color(gfc_plan* P, void* a, const float* rm, const float* rs) {
  const long long n = (long long)P->H * P->W;
  const int nblk = blocks_for(n), F = fields_of(P), L = launch_fields(P);
  const bool v4 = packed4(P, {a});
  float* sc = P->partial;
  for (int f0 = 0; f0 < F; f0 += L) {
    const int nf = F - f0 < L ? F - f0 : L;
    const dim3 g(nblk, nf);
    if (v4) k_moments_partial<T, 4><<<g, kThreads, 0, P->stream>>>((const T*)a, n, nblk, sc, f0);
    else k_moments_partial<T, 1><<<g, kThreads, 0, P->stream>>>((const T*)a, n, nblk, sc, f0);
    k_moments_finish<T><<<(nf + 7) / 8, 256, 0, P->stream>>>((const T*)a, n, nblk, sc, f0, nf, nullptr, nullptr);
    if (v4) k_color_apply<T, 4><<<g, kThreads, 0, P->stream>>>((T*)a, n, nblk, sc, f0, rm, rs);
    else k_color_apply<T, 1><<<g, kThreads, 0, P->stream>>>((T*)a, n, nblk, sc, f0, rm, rs);
  }
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

template <typename T>
gfc_status prepare_threshold(gfc_plan* P, const void* gx, const void* gy, float frac, float ref) {
  const long long n = (long long)P->H * P->W;
  const int nblk = blocks_for(n), F = fields_of(P), L = launch_fields(P);
  const bool v4 = packed4(P, {gx, gy});
  float* sc = P->partial;
  for (int f0 = 0; f0 < F; f0 += L) {
    const int nf = F - f0 < L ? F - f0 : L;
    const dim3 g(nblk, nf);
    if (!(ref > 0.f)) {
      if (v4) k_mag_max_partial<T, 4><<<g, kThreads, 0, P->stream>>>((const T*)gx, (const T*)gy, n, nblk, sc, f0);
      else k_mag_max_partial<T, 1><<<g, kThreads, 0, P->stream>>>((const T*)gx, (const T*)gy, n, nblk, sc, f0);
    }
    k_threshold_finish<<<(nf + 7) / 8, 256, 0, P->stream>>>(sc, nblk, f0, nf, frac, ref, P->edit_t2);
  }
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

template <typename T>
gfc_status run_threshold(gfc_plan* P, const void* gx, const void* gy, float frac, float ref, void* ox, void* oy) {
  if (gfc_status s = prepare_threshold<T>(P, gx, gy, frac, ref)) return s;
  const long long n = (long long)P->H * P->W;
  const int nblk = blocks_for(n), F = fields_of(P), L = launch_fields(P);
  const bool v4 = packed4(P, {gx, gy, ox, oy});
  for (int f0 = 0; f0 < F; f0 += L) {
    const int nf = F - f0 < L ? F - f0 : L;
    const dim3 g(nblk, nf);
    if (v4)
      k_threshold_apply<T, 4><<<g, kThreads, 0, P->stream>>>((const T*)gx, (const T*)gy, n, nblk, P->edit_t2, f0,
                                                              (T*)ox, (T*)oy);
    else
      k_threshold_apply<T, 1><<<g, kThreads, 0, P->stream>>>((const T*)gx, (const T*)gy, n, nblk, P->edit_t2, f0,
                                                              (T*)ox, (T*)oy);
  }
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

template <typename T>
gfc_status run_merge(gfc_plan* P, const void* gx, const void* gy, const void* edges, float alpha, void* ox, void* oy) {
  const long long total = (long long)fields_of(P) * P->H * P->W;
  const bool v4 = packed4(P, {gx, gy, edges, ox, oy});
  const long long packs = v4 ? total / 4 : total;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (packs + kThreads - 1) / kThreads;
  const long long cap = (long long)sms * 8;  // 8 resident blocks of 256 threads per SM
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (v4)
    k_merge<T, 4><<<(unsigned)blocks, kThreads, 0, P->stream>>>((const T*)gx, (const T*)gy, (const T*)edges, packs,
                                                                alpha, (T*)ox, (T*)oy);
  else
    k_merge<T, 1><<<(unsigned)blocks, kThreads, 0, P->stream>>>((const T*)gx, (const T*)gy, (const T*)edges, packs,
                                                                alpha, (T*)ox, (T*)oy);
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

template <typename T>
gfc_status run_ring(gfc_plan* P, const void* u, int ring, void* inner) {
  const int H = P->H, W = P->W;
  const long long nr = 2ll * ring * W + 2ll * ring * (H - 2 * ring);
  const int Hi = H - 2 * ring, Wi = W - 2 * ring;
  int rpb = kPerBlock / Wi;  // inner rows per block
  if (rpb < 1) rpb = 1;
  const int nbi = (Hi + rpb - 1) / rpb;
  const int nbr = blocks_for(nr * 4), F = fields_of(P), L = launch_fields(P);
  float* sc = P->partial;
  for (int f0 = 0; f0 < F; f0 += L) {
    const int nf = F - f0 < L ? F - f0 : L;
    k_ring_partial<T><<<dim3(nbr, nf), kThreads, 0, P->stream>>>((const T*)u, H, W, ring, nr, nbr, sc, f0);
    k_ring_apply<T><<<dim3(nbi, nf), kThreads, 0, P->stream>>>((const T*)u, H, W, ring, nr, nbr, rpb, sc, f0,
                                                              (T*)inner);
  }
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

}  // namespace

gfc_status gfc::edit_prepare_threshold(gfc_plan* P, const void* gx, const void* gy, float frac, float ref) {
  switch (P->dtype) {
    case GFC_F32: return prepare_threshold<float>(P, gx, gy, frac, ref);
    case GFC_F16: return prepare_threshold<__half>(P, gx, gy, frac, ref);
    default: return prepare_threshold<__nv_bfloat16>(P, gx, gy, frac, ref);
  }
}

#define GFC_DISPATCH(P, fn, ...)                                                     \
  ((P)->dtype == GFC_F32    ? fn<float>(P, __VA_ARGS__)                              \
   : (P)->dtype == GFC_F16  ? fn<__half>(P, __VA_ARGS__)                             \
                            : fn<__nv_bfloat16>(P, __VA_ARGS__))

extern "C" {

gfc_status gfc_field_stats(gfc_plan* plan, const void* fields, float* mean, float* std) {
  gfc::clear_error();
  if (gfc_status s = check_uniform(plan, "gfc_field_stats")) return s;
  if (!fields || !mean || !std) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_field_stats: null argument");
  if (mean == std) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_field_stats: mean and std alias");
  return GFC_DISPATCH(plan, run_moments, fields, mean, std);
}

gfc_status gfc_color_correct(gfc_plan* plan, void* out, const float* ref_mean, const float* ref_std) {
  gfc::clear_error();
  if (gfc_status s = check_uniform(plan, "gfc_color_correct")) return s;
  if (!out || !ref_mean || !ref_std) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_color_correct: null argument");
  return GFC_DISPATCH(plan, run_color, out, ref_mean, ref_std);
}

gfc_status gfc_gradient_threshold(gfc_plan* plan, const void* gx, const void* gy, float frac, float ref, void* gx_out,
                                  void* gy_out) {
  gfc::clear_error();
  if (gfc_status s = check_uniform(plan, "gfc_gradient_threshold")) return s;
  if (!gx || !gy || !gx_out || !gy_out)
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_gradient_threshold: null argument");
  if (!(frac >= 0.f) || !(ref == ref))
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_gradient_threshold: frac must be >= 0 and ref a number");
  if (gx_out == gy_out || gx_out == gy || gy_out == gx)
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_gradient_threshold: outputs alias each other or the other input");
  return GFC_DISPATCH(plan, run_threshold, gx, gy, frac, ref, gx_out, gy_out);
}

gfc_status gfc_gradient_merge(gfc_plan* plan, const void* gx, const void* gy, const void* edges, float alpha,
                              void* gx_out, void* gy_out) {
  gfc::clear_error();
  if (gfc_status s = check_uniform(plan, "gfc_gradient_merge")) return s;
  if (!gx || !gy || !edges || !gx_out || !gy_out)
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_gradient_merge: null argument");
  if (!(alpha >= 0.f && alpha <= 1.f)) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_gradient_merge: alpha outside [0, 1]");
  if (gx_out == gy_out || gx_out == gy || gy_out == gx || gx_out == edges || gy_out == edges)
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_gradient_merge: outputs alias each other or another input");
  return GFC_DISPATCH(plan, run_merge, gx, gy, edges, alpha, gx_out, gy_out);
}

gfc_status gfc_boundary_offset(gfc_plan* plan, const void* out, int ring, void* inner) {
  gfc::clear_error();
  if (gfc_status s = check_uniform(plan, "gfc_boundary_offset")) return s;
  if (!out || !inner) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_boundary_offset: null argument");
  if (ring < 1 || 2 * ring >= plan->H || 2 * ring >= plan->W)
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_boundary_offset: ring %d does not fit a %dx%d field", ring, plan->H,
                     plan->W);
  if (out == inner) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_boundary_offset: inner aliases out");
  return GFC_DISPATCH(plan, run_ring, out, ring, inner);
}

}  // extern "C"

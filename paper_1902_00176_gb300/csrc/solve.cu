// solve.cu -- the GFC solve (Eq. 23, Algorithm B) and its adjoint as three passes.
//
//   pass A  rows:    L = div E fused into the loads (Eq. 3), zero padding, real
//                    row transforms of length N, two rows per complex transform
//   pass B  columns: column transform of length M, multiply by the real Green
//                    spectrum G (Eq. 22), inverse column transform
//   pass C  rows:    inverse real row transforms, subtract u[0,0], crop the
//                    image block, cast to the storage dtype (Algorithm B)
//
// The spectrum between passes lives in the plan's scratch, [field][M][ldS]
// complex, of which only the Hermitian half (N/2+1 columns) is kept. Fields
// are processed in chunks sized so that one chunk's scratch stays in L2.
//
// Two real rows a, b share one complex transform: z = a + i b, Z = F(z), then
//   A[k] = (Z[k] + conj Z[N-k]) / 2,   B[k] = -i (Z[k] - conj Z[N-k]) / 2,
// and on the way back z = F^-1(A + i B) with the Hermitian extension of A and
// B, whose real and imaginary parts are the rows a and b.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "gfc_internal.h"

namespace gfc {

enum Mode { kGrad = 0, kLap = 1, kAdj = 2 };

struct PassArgs {
  int H, W, p, M, N, Nh, ldS;
  int nrows, ncols;  // support of pass A's input rows (from torus row/col p)
  int pairs;         // row pairs handled by the row pass
  int ppb;           // row pairs per block
  int nparts;        // pass A blocks per field (adjoint partial sums)
  FftPlan plan;      // the transform this pass runs
  // ragged batches: per-field sizes and offsets (nullptr for a uniform batch)
  const FieldDesc* fd;
  const FftPlan* plans;
};

// Load this block's field descriptor into A (ragged batches). pass: 0 row
// forward, 1 column, 2 row inverse. Returns false if the block has no work in
// its field (grids are sized for the largest field).
template <int MODE>
__device__ __forceinline__ bool ragged_field(PassArgs& A, int pass, FieldDesc& d) {
  d = A.fd[blockIdx.y];
  A.H = d.H; A.W = d.W; A.M = d.M; A.N = d.N; A.Nh = d.Nh; A.ldS = d.ldS; A.p = d.pad;
  A.nrows = (MODE == 0) ? d.H + 1 : d.H;
  A.ncols = (MODE == 0) ? d.W + 1 : d.W;
  const int pairs_in = (A.nrows + 1) / 2;
  A.nparts = (pairs_in + A.ppb - 1) / A.ppb;
  if (pass == 0) {
    A.plan = A.plans[2 * d.plan];
    A.pairs = pairs_in;
    return (int)blockIdx.x < A.nparts;
  }
  if (pass == 1) {
    A.plan = A.plans[2 * d.plan + 1];
    return (int)blockIdx.x * A.pairs < A.Nh;  // A.pairs carries the strip width here
  }
  A.plan = A.plans[2 * d.plan];
  A.pairs = (d.H + 1) / 2;
  return (int)blockIdx.x * A.ppb < A.pairs;
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T> __device__ __forceinline__ T from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_f<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename T>
__device__ __forceinline__ float ld(const T* __restrict__ g, int i, int j, int H, int W) {
  return (i >= 0 && i < H && j >= 0 && j < W) ? to_f(g[(size_t)i * W + j]) : 0.0f;
}

// Deterministic block sum: fixed per-thread order, fixed tree. All threads get the result.
__device__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float s = 0.0f;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// pass A
// ---------------------------------------------------------------------------
// EDIT (gradient mode only): the edit of Sec. 3.2.3 / Eq. 26 applied to every
// gradient value as it is loaded (edit_pixel), so the edited field is never stored.
template <typename T, int MODE, int EDIT = kEditNone>
__global__ void __launch_bounds__(256) k_pass_a(const T* __restrict__ in0, const T* __restrict__ in1,
                                                float2* __restrict__ spec, float* __restrict__ partial,
                                                const float2* __restrict__ twg, PassArgs A, EditArgs ed) {
  extern __shared__ float2 sm[];
  __shared__ float red[32];
  long long in_off = (long long)blockIdx.y * A.H * A.W, spec_off = (long long)blockIdx.y * A.M * A.ldS;
  if (A.fd) {
    FieldDesc d;
    if (!ragged_field<MODE>(A, 0, d)) return;
    in_off = d.in_off;
    spec_off = d.spec_off;
    twg += d.twN_off;
  }
  float2* tw = sm;
  float2* b0 = sm + A.N;
  float2* b1 = b0 + A.N;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const T* a = in0 + in_off;
  const T* b = (MODE == kGrad) ? in1 + in_off : nullptr;
  float2* S = spec + spec_off;
  for (int m = tid; m < A.N; m += nthr) tw[m] = twg[m];
  float acc = 0.0f;
  const int q0 = blockIdx.x * A.ppb;
  const int q1 = min(q0 + A.ppb, A.pairs);
  for (int q = q0; q < q1; ++q) {
    const int i0 = 2 * q, i1 = 2 * q + 1;
    const bool has1 = i1 < A.nrows;
    __syncthreads();
    for (int c = tid; c < A.N; c += nthr) {
      const int j = c - A.p;
      float va = 0.0f, vb = 0.0f;
      if (j >= 0 && j < A.ncols) {
        if (MODE == kGrad && EDIT != kEditNone) {
          const T* e = static_cast<const T*>(ed.edges) + (ed.edges ? in_off : 0);
          const float t2 = (EDIT == kEditThreshold) ? ed.t2[blockIdx.y] : 0.0f;
          const float2 c0 = edit_pixel<T, EDIT>(a, b, e, i0, j, A.H, A.W, t2, ed.alpha);
          va = c0.x - edit_pixel<T, EDIT>(a, b, e, i0, j - 1, A.H, A.W, t2, ed.alpha).x + c0.y -
               edit_pixel<T, EDIT>(a, b, e, i0 - 1, j, A.H, A.W, t2, ed.alpha).y;
          if (has1) {
            const float2 c1 = edit_pixel<T, EDIT>(a, b, e, i1, j, A.H, A.W, t2, ed.alpha);
            vb = c1.x - edit_pixel<T, EDIT>(a, b, e, i1, j - 1, A.H, A.W, t2, ed.alpha).x + c1.y - c0.y;
          }
        } else if (MODE == kGrad) {
          va = ld(a, i0, j, A.H, A.W) - ld(a, i0, j - 1, A.H, A.W) + ld(b, i0, j, A.H, A.W) - ld(b, i0 - 1, j, A.H, A.W);
          if (has1)
            vb = ld(a, i1, j, A.H, A.W) - ld(a, i1, j - 1, A.H, A.W) + ld(b, i1, j, A.H, A.W) - ld(b, i1 - 1, j, A.H, A.W);
        } else {
          va = ld(a, i0, j, A.H, A.W);
          if (has1) vb = ld(a, i1, j, A.H, A.W);
        }
      }
      if (MODE == kAdj) acc += va + vb;
      b0[c] = make_float2(va, vb);
    }
    __syncthreads();
    const float2* X = fft_smem<-1>(b0, b1, A.plan, 1, 1, tw, tid, nthr);
    for (int k = tid; k < A.Nh; k += nthr) {
      const float2 zk = X[k], zm = X[k == 0 ? 0 : A.N - k];
      S[(size_t)(A.p + i0) * A.ldS + k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      if (has1) S[(size_t)(A.p + i1) * A.ldS + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
  if (MODE == kAdj) {
    const float s = block_sum(acc, red);
    if (tid == 0) partial[(size_t)blockIdx.y * kMaxRowBlocks + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// pass B: S columns per block, interleaved in shared memory (element m of
// column f at m*S + f)
// ---------------------------------------------------------------------------
template <int S, int MODE>
__global__ void __launch_bounds__(256) k_pass_b(float2* __restrict__ spec, const float* __restrict__ G,
                                                const float2* __restrict__ twg, const float* __restrict__ partial,
                                                PassArgs A) {
  extern __shared__ float2 sm[];
  long long spec_off = (long long)blockIdx.y * A.M * A.ldS;
  if (A.fd) {
    FieldDesc d;
    A.pairs = S;
    if (!ragged_field<MODE>(A, 1, d)) return;
    spec_off = d.spec_off;
    twg += d.twM_off;
    G += d.G_off;
  }
  float2* tw = sm;
  float2* b0 = sm + A.M;
  float2* b1 = b0 + (size_t)A.M * S;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int l0 = blockIdx.x * S;
  float2* Sp = spec + spec_off;
  for (int m = tid; m < A.M; m += nthr) tw[m] = twg[m];
  float tot = 0.0f;
  if (MODE == kAdj) {
    const float* pp = partial + (size_t)blockIdx.y * kMaxRowBlocks;
    for (int i = 0; i < A.nparts; ++i) tot += pp[i];
  }
  for (int t = tid; t < A.M * S; t += nthr) {
    const int f = t % S, r = t / S, l = l0 + f;
    float2 v = make_float2(0.0f, 0.0f);
    if (l < A.Nh) {
      if (r >= A.p && r < A.p + A.nrows) v = Sp[(size_t)r * A.ldS + l];
      else if (MODE == kAdj && r == 0) v = make_float2(-tot, 0.0f);  // row DFT of -(sum) e_00
    }
    b0[t] = v;
  }
  __syncthreads();
  float2* X = fft_smem<-1>(b0, b1, A.plan, S, S, tw, tid, nthr);
  float2* Y = (X == b0) ? b1 : b0;
  for (int t = tid; t < A.M * S; t += nthr) {
    const int f = t % S, k = t / S, l = l0 + f;
    const float g = (l < A.Nh) ? G[(size_t)k * A.Nh + l] : 0.0f;
    X[t] = cscale(X[t], g);
  }
  __syncthreads();
  const float2* Z = fft_smem<+1>(X, Y, A.plan, S, S, tw, tid, nthr);
  for (int t = tid; t < A.M * S; t += nthr) {
    const int f = t % S, r = t / S, l = l0 + f;
    if (l >= A.Nh) continue;
    const bool keep = (MODE == kAdj) ? (r >= A.p && r <= A.p + A.H) : (r == 0 || (r >= A.p && r < A.p + A.H));
    if (keep) Sp[(size_t)r * A.ldS + l] = Z[t];
  }
}

// ---------------------------------------------------------------------------
// pass C
// ---------------------------------------------------------------------------
// Build z = A + i B over the full length N from Hermitian halves of rows ra, rb
// (rb < 0: zero row). The imaginary parts of bins 0 and N/2 are dropped, as a
// real inverse transform does.
__device__ __forceinline__ void load_pair_hermitian(const float2* __restrict__ Sp, int ldS, int N, int ra, int rb,
                                                    float2* __restrict__ dst, int tid, int nthr) {
  const int half = N / 2;
  for (int l = tid; l < N; l += nthr) {
    const bool lo = l <= half;
    const int src = lo ? l : N - l;
    float2 ya = Sp[(size_t)ra * ldS + src];
    float2 yb = rb >= 0 ? Sp[(size_t)rb * ldS + src] : make_float2(0.0f, 0.0f);
    if (src == 0 || src == half) { ya.y = 0.0f; yb.y = 0.0f; }
    dst[l] = lo ? make_float2(ya.x - yb.y, ya.y + yb.x) : make_float2(ya.x + yb.y, yb.x - ya.y);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pass_c(const float2* __restrict__ spec, T* __restrict__ out,
                                                const float2* __restrict__ twg, PassArgs A) {
  extern __shared__ float2 sm[];
  __shared__ double redd[32];
  long long out_off = (long long)blockIdx.y * A.H * A.W, spec_off = (long long)blockIdx.y * A.M * A.ldS;
  if (A.fd) {
    FieldDesc d;
    if (!ragged_field<kGrad>(A, 2, d)) return;
    out_off = d.in_off;
    spec_off = d.spec_off;
    twg += d.twN_off;
  }
  float2* tw = sm;
  float2* b0 = sm + A.N;
  float2* b1 = b0 + A.N;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float2* Sp = spec + spec_off;
  T* o = out + out_off;
  for (int m = tid; m < A.N; m += nthr) tw[m] = twg[m];
  // u[0,0] = sum over the full row-0 spectrum = Re Y[0] + Re Y[N/2] + 2 sum_{0<l<N/2} Re Y[l],
  // accumulated in FP64 (an error in u[0,0] shifts every output pixel)
  double s = 0.0;
  for (int l = tid; l <= A.N / 2; l += nthr) {
    const double x = Sp[l].x;
    s += (l == 0 || l == A.N / 2) ? x : 2.0 * x;
  }
  const float u00 = (float)block_sum_d(s, redd);
  const int q0 = blockIdx.x * A.ppb;
  const int q1 = min(q0 + A.ppb, A.pairs);
  for (int q = q0; q < q1; ++q) {
    const int i0 = 2 * q, i1 = 2 * q + 1;
    const bool has1 = i1 < A.H;
    __syncthreads();
    load_pair_hermitian(Sp, A.ldS, A.N, A.p + i0, has1 ? A.p + i1 : -1, b0, tid, nthr);
    __syncthreads();
    const float2* Z = fft_smem<+1>(b0, b1, A.plan, 1, 1, tw, tid, nthr);
    for (int j = tid; j < A.W; j += nthr) {
      const float2 z = Z[A.p + j];
      o[(size_t)i0 * A.W + j] = from_f<T>(z.x - u00);
      if (has1) o[(size_t)i1 * A.W + j] = from_f<T>(z.y - u00);
    }
  }
}

// Adjoint pass C: w rows 0..H (torus p..p+H) come back from pass B; the
// transpose of the divergence gives
//   grad_gx[i,j] = w[i,j] - w[i,j+1],   grad_gy[i,j] = w[i,j] - w[i+1,j].
// A block owns output rows [2 q0, 2 q1) and also transforms pair q1 to get the
// row below its last one.
template <typename T>
__global__ void __launch_bounds__(256) k_pass_c_adj(const float2* __restrict__ spec, T* __restrict__ ggx,
                                                    T* __restrict__ ggy, const float2* __restrict__ twg,
                                                    PassArgs A) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + A.N;
  float2* b1 = b0 + A.N;
  const int tid = threadIdx.x, nthr = blockDim.x;
  long long out_off = (long long)blockIdx.y * A.H * A.W, spec_off = (long long)blockIdx.y * A.M * A.ldS;
  if (A.fd) {
    FieldDesc d;
    if (!ragged_field<kAdj>(A, 2, d)) return;
    out_off = d.in_off;
    spec_off = d.spec_off;
    twg += d.twN_off;
    tw = sm;
    b0 = sm + A.N;
    b1 = b0 + A.N;
  }
  float* prev = reinterpret_cast<float*>(b1 + A.N);  // [W] row 2q-1 of w from the previous pair
  const float2* Sp = spec + spec_off;
  T* gx = ggx + out_off;
  T* gy = ggy + out_off;
  for (int m = tid; m < A.N; m += nthr) tw[m] = twg[m];
  const int q0 = blockIdx.x * A.ppb;
  const int q1 = min(q0 + A.ppb, A.pairs);
  const int wrows = A.H + 1;
  for (int q = q0; q <= q1; ++q) {
    const int i0 = 2 * q, i1 = 2 * q + 1;
    if (i0 >= wrows) break;
    const bool has1 = i1 < wrows;
    __syncthreads();
    load_pair_hermitian(Sp, A.ldS, A.N, A.p + i0, has1 ? A.p + i1 : -1, b0, tid, nthr);
    __syncthreads();
    const float2* Z = fft_smem<+1>(b0, b1, A.plan, 1, 1, tw, tid, nthr);
    for (int j = tid; j < A.W; j += nthr) {
      const float2 z = Z[A.p + j], zr = Z[A.p + j + 1];
      if (q > q0 && i0 - 1 < A.H) gy[(size_t)(i0 - 1) * A.W + j] = from_f<T>(prev[j] - z.x);
      if (q < q1) {
        if (i0 < A.H) {
          gx[(size_t)i0 * A.W + j] = from_f<T>(z.x - zr.x);
          gy[(size_t)i0 * A.W + j] = from_f<T>(z.x - z.y);
        }
        if (i1 < A.H) gx[(size_t)i1 * A.W + j] = from_f<T>(z.y - zr.y);
        prev[j] = z.y;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// standalone batched complex transform (test entry point)
// ---------------------------------------------------------------------------
template <int DIR>
__global__ void __launch_bounds__(256) k_fft_rows(const float2* __restrict__ in, float2* __restrict__ out,
                                                  FftPlan pl) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + pl.n;
  float2* b1 = b0 + pl.n;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int m = tid; m < pl.n; m += nthr) {
    double s, c;
    sincospi(2.0 * (double)m / (double)pl.n, &s, &c);
    tw[m] = make_float2((float)c, (float)(-s));
  }
  const size_t row = blockIdx.x;
  for (int m = tid; m < pl.n; m += nthr) b0[m] = in[row * pl.n + m];
  __syncthreads();
  const float2* X = fft_smem<DIR>(b0, b1, pl, 1, 1, tw, tid, nthr);
  for (int m = tid; m < pl.n; m += nthr) out[row * pl.n + m] = X[m];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Raise a kernel's dynamic shared-memory cap to at least `smem`. The cap is
// tracked per kernel function (several launch sites share a kernel) and is
// never lowered, since a launch above the current cap is rejected.
struct SmemCap {
  const void* fn;
  int bytes;
};
static SmemCap g_smem_caps[256];
static int g_smem_ncaps = 0;
static std::mutex g_smem_mu;

template <typename K>
static cudaError_t ensure_smem(K kernel, size_t smem) {
  const void* fn = reinterpret_cast<const void*>(kernel);
  std::lock_guard<std::mutex> lock(g_smem_mu);
  int i = 0;
  for (; i < g_smem_ncaps; ++i)
    if (g_smem_caps[i].fn == fn) break;
  if (i < g_smem_ncaps && (int)smem <= g_smem_caps[i].bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (i == g_smem_ncaps) {
    if (g_smem_ncaps == 256) return cudaSuccess;  // table full: the attribute is still set for this launch
    g_smem_caps[g_smem_ncaps++] = SmemCap{fn, (int)smem};
  } else {
    g_smem_caps[i].bytes = (int)smem;
  }
  return cudaSuccess;
}

void prof_begin(gfc_plan* P, int pass, cudaStream_t st) {
  P->prof.launches[pass] += 1;
  if (!P->profiling) return;
  if (P->ev_used >= P->ev_cap) {
    P->prof.dropped += 1;
    return;
  }
  P->ev_pass[P->ev_used] = pass;
  cudaEventRecord(P->ev_start[P->ev_used], st);
}

void prof_end(gfc_plan* P, cudaStream_t st) {
  if (!P->profiling || P->ev_used >= P->ev_cap) return;
  cudaEventRecord(P->ev_stop[P->ev_used], st);
  P->ev_used += 1;
}

static int pick_strip(int M) {
  // columns per pass-B block: largest power of two with (M + 2 M S) * 8 B <= 200 KB
  for (int S = 8; S > 1; S >>= 1)
    if ((size_t)(M + 2 * M * S) * sizeof(float2) <= 200u * 1024u) return S;
  return 1;
}

static PassArgs base_args(const gfc_plan* P) {
  PassArgs a;
  a.H = P->H; a.W = P->W; a.p = P->pad; a.M = P->M; a.N = P->N; a.Nh = P->Nh; a.ldS = P->ldS;
  a.nrows = a.ncols = a.pairs = a.ppb = a.nparts = 0;
  a.plan = P->rowplan;
  a.fd = nullptr;
  a.plans = nullptr;
  return a;
}

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

template <int S, int MODE>
static cudaError_t launch_b(gfc_plan* P, const Bufs& bf, PassArgs B, int nf, cudaStream_t st) {
  const size_t smem = (size_t)(P->M + 2 * (size_t)P->M * S) * sizeof(float2);
  auto k = k_pass_b<S, MODE>;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  prof_begin(P, 1, st);
  k<<<dim3(ceil_div(P->Nh, S), nf), 256, smem, st>>>(bf.spec, P->G, P->twM, bf.partial, B);
  prof_end(P, st);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_b_any(gfc_plan* P, const Bufs& bf, PassArgs B, int nf, cudaStream_t st) {
  switch (pick_strip(P->M)) {
    case 8: return launch_b<8, MODE>(P, bf, B, nf, st);
    case 4: return launch_b<4, MODE>(P, bf, B, nf, st);
    case 2: return launch_b<2, MODE>(P, bf, B, nf, st);
    default: return launch_b<1, MODE>(P, bf, B, nf, st);
  }
}

template <typename T, int MODE>
static cudaError_t run_chunk(gfc_plan* P, const Bufs& bf, const T* in0, const T* in1, T* out0, T* out1, int nf,
                             cudaStream_t st, const EditArgs* ed = nullptr) {
  if (P->exact) return run_chunk_exact(P, bf, MODE, in0, in1, out0, out1, nf, st, ed);
  if (P->fast) {  // register-resident passes; the generic ones serve what they do not cover
    const cudaError_t e = run_chunk_fast(P, bf, MODE, in0, in1, out0, out1, nf, st, ed);
    if (e != cudaErrorNotSupported) return e;
  }
  const EditArgs none{kEditNone, 0.0f, nullptr, nullptr, nullptr, nullptr};
  const EditArgs& E = ed ? *ed : none;
  // pass A
  PassArgs A = base_args(P);
  A.nrows = (MODE == kGrad) ? P->H + 1 : P->H;
  A.ncols = (MODE == kGrad) ? P->W + 1 : P->W;
  A.pairs = ceil_div(A.nrows, 2);
  A.ppb = 4;
  if (ceil_div(A.pairs, A.ppb) > kMaxRowBlocks) A.ppb = ceil_div(A.pairs, kMaxRowBlocks);
  A.nparts = ceil_div(A.pairs, A.ppb);
  cudaError_t e;
  {
      const size_t smem = 3 * (size_t)P->N * sizeof(float2);
    auto k = k_pass_a<T, MODE>;
    if constexpr (MODE == kGrad) {
      if (E.kind == kEditThreshold) k = k_pass_a<T, MODE, kEditThreshold>;
      if (E.kind == kEditMerge) k = k_pass_a<T, MODE, kEditMerge>;
    }
    if ((e = ensure_smem(k, smem)) != cudaSuccess) return e;
    prof_begin(P, 0, st);
    k<<<dim3(A.nparts, nf), 256, smem, st>>>(in0, in1, bf.spec, bf.partial, P->twN, A, E);
    prof_end(P, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // pass B
  PassArgs B = A;
  B.plan = P->colplan;
  if ((e = launch_b_any<MODE>(P, bf, B, nf, st)) != cudaSuccess) return e;
  // pass C
  PassArgs C = base_args(P);
  C.ppb = 4;
  C.pairs = ceil_div(P->H, 2);
  if (MODE == kAdj) {
      const size_t smem = 3 * (size_t)P->N * sizeof(float2) + (size_t)P->W * sizeof(float);
    auto k = k_pass_c_adj<T>;
    if ((e = ensure_smem(k, smem)) != cudaSuccess) return e;
    prof_begin(P, 2, st);
    k<<<dim3(ceil_div(C.pairs, C.ppb), nf), 256, smem, st>>>(bf.spec, out0, out1, P->twN, C);
    prof_end(P, st);
  } else {
      const size_t smem = 3 * (size_t)P->N * sizeof(float2);
    auto k = k_pass_c<T>;
    if ((e = ensure_smem(k, smem)) != cudaSuccess) return e;
    prof_begin(P, 2, st);
    k<<<dim3(ceil_div(C.pairs, C.ppb), nf), 256, smem, st>>>(bf.spec, out0, P->twN, C);
    prof_end(P, st);
  }
  return cudaGetLastError();
}

// Chunk c runs on slot c mod nslots: its own scratch and internal stream, forked
// from the plan's stream and joined back into it at the end of the call.
template <typename T, int MODE>
static gfc_status run_all(gfc_plan* P, const void* a, const void* b, void* o0, void* o1,
                          const EditArgs* ed = nullptr) {
  const long fields = (long)P->batch * P->C;
  const size_t fe = (size_t)P->H * P->W;
  P->prof.calls += 1;
  const bool fork = P->nslots > 1;
  if (fork) {
    GFC_CUDA_TRY(cudaEventRecord(P->ev_fork, P->stream));
    for (int s = 0; s < P->nslots; ++s) GFC_CUDA_TRY(cudaStreamWaitEvent(P->slot_stream[s], P->ev_fork, 0));
  }
  long c = 0;
  for (long f0 = 0; f0 < fields; f0 += P->chunk, ++c) {
    const int nf = (int)((fields - f0 < P->chunk) ? fields - f0 : P->chunk);
    const T* in0 = static_cast<const T*>(a) + f0 * fe;
    const T* in1 = b ? static_cast<const T*>(b) + f0 * fe : nullptr;
    T* out0 = static_cast<T*>(o0) + f0 * fe;
    T* out1 = o1 ? static_cast<T*>(o1) + f0 * fe : nullptr;
    const int s = fork ? (int)(c % P->nslots) : 0;
    EditArgs ec{kEditNone, 0.0f, nullptr, nullptr, nullptr, nullptr};
    if (ed) {  // the edit's per-field data, at this chunk's first field
      ec = *ed;
      if (ec.edges) ec.edges = static_cast<const T*>(ec.edges) + f0 * fe;
      if (ec.t2) ec.t2 += f0;
      if (ec.ref_mean) {
        ec.ref_mean += f0;
        ec.ref_std += f0;
      }
    }
    cudaError_t e = run_chunk<T, MODE>(P, slot_bufs(P, s), in0, in1, out0, out1, nf,
                                       fork ? P->slot_stream[s] : P->stream, ed ? &ec : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "gfc solve launch");
  }
  if (fork) {
    for (int s = 0; s < P->nslots; ++s) {
      GFC_CUDA_TRY(cudaEventRecord(P->slot_done[s], P->slot_stream[s]));
      GFC_CUDA_TRY(cudaStreamWaitEvent(P->stream, P->slot_done[s], 0));
    }
  }
  return GFC_OK;
}

// Ragged batches: per chunk of fields, each pass is one launch over all its
// fields; every block reads its field's descriptor (sizes, table offsets,
// schedules) and grids are sized for the largest field.
template <typename T, int MODE>
static gfc_status run_ragged(gfc_plan* P, const void* a, const void* b, void* o0, void* o1) {
  cudaStream_t st = P->stream;
  P->prof.calls += 1;
  const int nrows_max = (MODE == kGrad) ? P->maxH + 1 : P->maxH;
  const int pairs_max = (nrows_max + 1) / 2;
  int ppb = 4;
  if (ceil_div(pairs_max, ppb) > kMaxRowBlocks) ppb = ceil_div(pairs_max, kMaxRowBlocks);
  const int S = pick_strip(P->maxM);
  for (int c = 0; c < P->nchunks; ++c) {
    const int f0 = P->chunk_begin[c], nf = P->chunk_begin[c + 1] - f0;
    PassArgs A = base_args(P);
    A.M = P->maxM;
    A.N = P->maxN;
    A.ppb = ppb;
    A.fd = P->d_desc + f0;
    A.plans = P->d_plans;
    cudaError_t e;
    {
      const size_t smem = 3 * (size_t)P->maxN * sizeof(float2);
      auto k = k_pass_a<T, MODE>;
      if ((e = ensure_smem(k, smem)) != cudaSuccess) return cuda_fail(e, "gfc ragged pass A");
      prof_begin(P, 0, st);
      k<<<dim3(ceil_div(pairs_max, ppb), nf), 256, smem, st>>>(static_cast<const T*>(a), static_cast<const T*>(b),
                                                                 P->spec, P->partial, P->twN, A,
                                                                 EditArgs{kEditNone, 0.0f, nullptr, nullptr, nullptr, nullptr});
      prof_end(P, st);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gfc ragged pass A");
    }
    {
      const size_t smem = (size_t)(P->maxM + 2 * (size_t)P->maxM * S) * sizeof(float2);
      const dim3 grid(ceil_div(P->maxNh, S), nf);
      prof_begin(P, 1, st);
      switch (S) {
        case 8:
          if ((e = ensure_smem(k_pass_b<8, MODE>, smem)) != cudaSuccess) break;
          k_pass_b<8, MODE><<<grid, 256, smem, st>>>(P->spec, P->G, P->twN, P->partial, A);
          break;
        case 4:
          if ((e = ensure_smem(k_pass_b<4, MODE>, smem)) != cudaSuccess) break;
          k_pass_b<4, MODE><<<grid, 256, smem, st>>>(P->spec, P->G, P->twN, P->partial, A);
          break;
        case 2:
          if ((e = ensure_smem(k_pass_b<2, MODE>, smem)) != cudaSuccess) break;
          k_pass_b<2, MODE><<<grid, 256, smem, st>>>(P->spec, P->G, P->twN, P->partial, A);
          break;
        default:
          if ((e = ensure_smem(k_pass_b<1, MODE>, smem)) != cudaSuccess) break;
          k_pass_b<1, MODE><<<grid, 256, smem, st>>>(P->spec, P->G, P->twN, P->partial, A);
      }
      prof_end(P, st);
      if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gfc ragged pass B");
    }
    {
      const int pairs_out = (P->maxH + 1) / 2;
      const dim3 grid(ceil_div(pairs_out, ppb), nf);
      prof_begin(P, 2, st);
      if (MODE == kAdj) {
        const size_t smem = 3 * (size_t)P->maxN * sizeof(float2) + (size_t)P->maxW * sizeof(float);
        if ((e = ensure_smem(k_pass_c_adj<T>, smem)) == cudaSuccess)
          k_pass_c_adj<T><<<grid, 256, smem, st>>>(P->spec, static_cast<T*>(o0), static_cast<T*>(o1), P->twN, A);
      } else {
        const size_t smem = 3 * (size_t)P->maxN * sizeof(float2);
        if ((e = ensure_smem(k_pass_c<T>, smem)) == cudaSuccess)
          k_pass_c<T><<<grid, 256, smem, st>>>(P->spec, static_cast<T*>(o0), P->twN, A);
      }
      prof_end(P, st);
      if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gfc ragged pass C");
    }
  }
  return GFC_OK;
}

template <int MODE>
static gfc_status dispatch(gfc_plan* P, const void* a, const void* b, void* o0, void* o1,
                           const EditArgs* ed = nullptr);

// A ragged plan's sub-plans (one per item on the register-resident passes), each
// on its internal stream, forked from and joined into the plan's stream; the
// generic part runs on the plan's stream meanwhile.
template <int MODE>
static gfc_status run_ragged_subplans(gfc_plan* P, const void* a, const void* b, void* o0, void* o1) {
  const size_t es = dtype_size(P->dtype);
  auto at = [&](const void* base, long long off) -> const void* {
    return base ? static_cast<const char*>(base) + off * (long long)es : nullptr;
  };
  GFC_CUDA_TRY(cudaEventRecord(P->rag_fork, P->stream));
  for (int s = 0; s < P->rag_active; ++s) GFC_CUDA_TRY(cudaStreamWaitEvent(P->rag_stream[s], P->rag_fork, 0));
  for (int j = 0; j < P->nsub; ++j) {
    gfc_plan* Q = P->sub[j];
    Q->stream = P->rag_stream[P->sub_stream[j]];
    const long long off = P->sub_off[j];
    gfc_status st = dispatch<MODE>(Q, at(a, off), at(b, off), const_cast<void*>(at(o0, off)),
                                   const_cast<void*>(at(o1, off)));
    if (st != GFC_OK) return st;
  }
  for (int s = 0; s < P->rag_active; ++s) {
    GFC_CUDA_TRY(cudaEventRecord(P->rag_done[s], P->rag_stream[s]));
    GFC_CUDA_TRY(cudaStreamWaitEvent(P->stream, P->rag_done[s], 0));
  }
  return GFC_OK;
}

template <int MODE>
static gfc_status dispatch(gfc_plan* P, const void* a, const void* b, void* o0, void* o1, const EditArgs* ed) {
  if (P->ragged) {
    if (P->nsub) {
      P->prof.calls += 1;
      if (gfc_status st = run_ragged_subplans<MODE>(P, a, b, o0, o1)) return st;
      if (P->nfields == 0) return GFC_OK;
    }
    switch (P->dtype) {
      case GFC_F32: return run_ragged<float, MODE>(P, a, b, o0, o1);
      case GFC_F16: return run_ragged<__half, MODE>(P, a, b, o0, o1);
      default: return run_ragged<__nv_bfloat16, MODE>(P, a, b, o0, o1);
    }
  }
  switch (P->dtype) {
    case GFC_F32: return run_all<float, MODE>(P, a, b, o0, o1, ed);
    case GFC_F16: return run_all<__half, MODE>(P, a, b, o0, o1, ed);
    default: return run_all<__nv_bfloat16, MODE>(P, a, b, o0, o1, ed);
  }
}

static bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

// Host-buffer pipeline: chunk c uses staging buffer c % 2. copy_in waits until
// the solve of chunk c-2 has consumed that buffer's inputs, the compute stream
// waits for the inputs and for the copy-out of chunk c-2 to free the output
// buffer, copy_out waits for the solve.
static gfc_status host_setup(gfc_plan* P) {
  if (P->host_ready) return GFC_OK;
  // Host<->device copies (about 210 GB/s in, 190 GB/s out on the GB300's link,
  // 340 GB/s both ways at once) bound this path, so the batch is cut into
  // steps whose copies in both directions overlap the solves of the others;
  // more steps shorten the unoverlapped first copy-in and last copy-out.
  // Measured on 100 x 801x1200 fields: 32 steps over 3 rotating buffers, 21.8k
  // solves/s; 8 steps over 2 buffers, 20.4k.
  const long fields = (long)P->batch * P->C;
  const int steps = 32, nb = 3;
  long hc = (fields + steps - 1) / steps;
  if (hc > P->chunk) hc = P->chunk;
  if (hc < 1) hc = 1;
  P->host_chunk = (int)hc;
  P->host_bufs = nb;
  const size_t bytes = (size_t)hc * P->H * P->W * dtype_size(P->dtype);
  for (int b = 0; b < nb; ++b) {
    GFC_CUDA_TRY(cudaMalloc(&P->stage_in[b][0], bytes));
    GFC_CUDA_TRY(cudaMalloc(&P->stage_in[b][1], bytes));
    GFC_CUDA_TRY(cudaMalloc(&P->stage_out[b], bytes));
    GFC_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_in[b], cudaEventDisableTiming));
    GFC_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_comp[b], cudaEventDisableTiming));
    GFC_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_out[b], cudaEventDisableTiming));
  }
  GFC_CUDA_TRY(cudaStreamCreateWithFlags(&P->copy_in, cudaStreamNonBlocking));
  GFC_CUDA_TRY(cudaStreamCreateWithFlags(&P->copy_out, cudaStreamNonBlocking));
  P->host_ready = true;
  return GFC_OK;
}

template <typename T>
static gfc_status run_host(gfc_plan* P, const void* gx, const void* gy, void* out) {
  gfc_status st = host_setup(P);
  if (st != GFC_OK) return st;
  const long fields = (long)P->batch * P->C;
  const size_t fe = (size_t)P->H * P->W;
  cudaStream_t cs = P->stream;
  // the copy streams start after everything already queued on the plan's stream
  cudaEvent_t start = P->ev_comp[1];
  GFC_CUDA_TRY(cudaEventRecord(start, cs));
  GFC_CUDA_TRY(cudaStreamWaitEvent(P->copy_in, start, 0));
  GFC_CUDA_TRY(cudaStreamWaitEvent(P->copy_out, start, 0));
  P->prof.calls += 1;
  long c = 0;
  const int hc = P->host_chunk, nb = P->host_bufs;
  for (long f0 = 0; f0 < fields; f0 += hc, ++c) {
    const int b = (int)(c % nb);
    const int nf = (int)((fields - f0 < hc) ? fields - f0 : hc);
    const size_t bytes = (size_t)nf * fe * sizeof(T);
    // buffer b is free for copy-in once the solve of step c - nb has read it
    if (c >= nb) GFC_CUDA_TRY(cudaStreamWaitEvent(P->copy_in, P->ev_comp[b], 0));
    GFC_CUDA_TRY(cudaMemcpyAsync(P->stage_in[b][0], static_cast<const T*>(gx) + f0 * fe, bytes,
                                 cudaMemcpyHostToDevice, P->copy_in));
    GFC_CUDA_TRY(cudaMemcpyAsync(P->stage_in[b][1], static_cast<const T*>(gy) + f0 * fe, bytes,
                                 cudaMemcpyHostToDevice, P->copy_in));
    GFC_CUDA_TRY(cudaEventRecord(P->ev_in[b], P->copy_in));
    GFC_CUDA_TRY(cudaStreamWaitEvent(cs, P->ev_in[b], 0));
    // ... and its output buffer once the copy-out of step c - nb is done
    if (c >= nb) GFC_CUDA_TRY(cudaStreamWaitEvent(cs, P->ev_out[b], 0));
    cudaError_t e = run_chunk<T, kGrad>(P, slot_bufs(P, 0), static_cast<const T*>(P->stage_in[b][0]),
                                        static_cast<const T*>(P->stage_in[b][1]), static_cast<T*>(P->stage_out[b]),
                                        nullptr, nf, cs);
    if (e != cudaSuccess) return cuda_fail(e, "gfc host solve launch");
    GFC_CUDA_TRY(cudaEventRecord(P->ev_comp[b], cs));
    GFC_CUDA_TRY(cudaStreamWaitEvent(P->copy_out, P->ev_comp[b], 0));
    GFC_CUDA_TRY(cudaMemcpyAsync(static_cast<T*>(out) + f0 * fe, P->stage_out[b], bytes, cudaMemcpyDeviceToHost,
                                 P->copy_out));
    GFC_CUDA_TRY(cudaEventRecord(P->ev_out[b], P->copy_out));
  }
  // the plan's stream completes only after the last copy-out (copy-outs run in order)
  GFC_CUDA_TRY(cudaStreamWaitEvent(cs, P->ev_out[(int)((c - 1) % nb)], 0));
  return GFC_OK;
}

void release_host_state(gfc_plan* P) {
  if (P->host_ready) {
    for (int b = 0; b < P->host_bufs; ++b) {
      cudaFree(P->stage_in[b][0]);
      cudaFree(P->stage_in[b][1]);
      cudaFree(P->stage_out[b]);
      cudaEventDestroy(P->ev_in[b]);
      cudaEventDestroy(P->ev_comp[b]);
      cudaEventDestroy(P->ev_out[b]);
    }
    cudaStreamDestroy(P->copy_in);
    cudaStreamDestroy(P->copy_out);
    P->host_ready = false;
  }
  if (P->ev_cap) {
    for (int i = 0; i < P->ev_cap; ++i) {
      cudaEventDestroy(P->ev_start[i]);
      cudaEventDestroy(P->ev_stop[i]);
    }
    free(P->ev_start);
    free(P->ev_stop);
    free(P->ev_pass);
    P->ev_cap = P->ev_used = 0;
  }
}

}  // namespace gfc

using namespace gfc;

extern "C" {

gfc_status gfc_solve_from_gradient(gfc_plan* plan, const void* gx, const void* gy, void* out) {
  clear_error();
  if (!plan || !gx || !gy || !out) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient: null argument");
  if (misaligned(gx) || misaligned(gy) || misaligned(out))
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient: pointers must be 16-byte aligned");
  if (out == gx || out == gy) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient: out aliases an input");
  return dispatch<kGrad>(plan, gx, gy, out, nullptr);
}

}  // extern "C"

// Validate `edit` and turn it into the passes' EditArgs (the threshold's per-field
// squared thresholds prepared in the plan's scratch).
static gfc_status prepare_edit(gfc_plan* plan, const void* gx, const void* gy, const gfc_edit* edit, EditArgs* ed,
                               const char* who) {
  *ed = EditArgs{kEditNone, 0.0f, nullptr, nullptr, nullptr, nullptr};
  if (!edit || edit->kind == GFC_EDIT_NONE) return GFC_OK;
  if (plan->ragged) return fail(GFC_ERR_UNSUPPORTED, "%s: ragged plans are not supported", who);
  if (edit->kind == GFC_EDIT_THRESHOLD) {
    if (!(edit->frac >= 0.0f) || !(edit->ref == edit->ref))
      return fail(GFC_ERR_INVALID_ARG, "%s: frac must be >= 0 and ref a number", who);
    if (gfc_status s = edit_prepare_threshold(plan, gx, gy, edit->frac, edit->ref)) return s;
    ed->kind = kEditThreshold;
    ed->t2 = plan->edit_t2;
  } else if (edit->kind == GFC_EDIT_MERGE) {
    if (!edit->edges) return fail(GFC_ERR_INVALID_ARG, "%s: merge needs an edge map", who);
    if (!(edit->alpha >= 0.0f && edit->alpha <= 1.0f)) return fail(GFC_ERR_INVALID_ARG, "%s: alpha outside [0, 1]", who);
    ed->kind = kEditMerge;
    ed->alpha = edit->alpha;
    ed->edges = edit->edges;
  } else {
    return fail(GFC_ERR_INVALID_ARG, "%s: unknown edit kind %d", who, edit->kind);
  }
  return GFC_OK;
}

extern "C" {

gfc_status gfc_solve_edited(gfc_plan* plan, const void* gx, const void* gy, const gfc_edit* edit, void* out) {
  clear_error();
  if (!plan || !gx || !gy || !edit || !out) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_edited: null argument");
  if (misaligned(gx) || misaligned(gy) || misaligned(out))
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_edited: pointers must be 16-byte aligned");
  if (out == gx || out == gy || out == edit->edges)
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_edited: out aliases an input");
  if (edit->kind == GFC_EDIT_NONE) return dispatch<kGrad>(plan, gx, gy, out, nullptr);
  EditArgs ed;
  if (gfc_status s = prepare_edit(plan, gx, gy, edit, &ed, "gfc_solve_edited")) return s;
  return dispatch<kGrad>(plan, gx, gy, out, nullptr, &ed);
}

gfc_status gfc_solve_corrected(gfc_plan* plan, const void* gx, const void* gy, const gfc_edit* edit,
                               const float* ref_mean, const float* ref_std, void* out) {
  clear_error();
  if (!plan || !gx || !gy || !ref_mean || !ref_std || !out)
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_corrected: null argument");
  if (misaligned(gx) || misaligned(gy) || misaligned(out))
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_corrected: pointers must be 16-byte aligned");
  if (out == gx || out == gy || (edit && out == edit->edges))
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_corrected: out aliases an input");
  if (plan->ragged) return fail(GFC_ERR_UNSUPPORTED, "gfc_solve_corrected: ragged plans are not supported");
  if (plan->fast && plan->tri && !plan->exact) {
    EditArgs ed;
    if (gfc_status s = prepare_edit(plan, gx, gy, edit, &ed, "gfc_solve_corrected")) return s;
    ed.ref_mean = ref_mean;
    ed.ref_std = ref_std;
    return dispatch<kGrad>(plan, gx, gy, out, nullptr, &ed);
  }
  // other plans: the solve, then the separate statistics and correction passes
  gfc_status s = (edit && edit->kind != GFC_EDIT_NONE) ? gfc_solve_edited(plan, gx, gy, edit, out)
                                                       : gfc_solve_from_gradient(plan, gx, gy, out);
  if (s != GFC_OK) return s;
  return gfc_color_correct(plan, out, ref_mean, ref_std);
}

gfc_status gfc_solve_from_laplacian(gfc_plan* plan, const void* lap, void* out) {
  clear_error();
  if (!plan || !lap || !out) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_laplacian: null argument");
  if (misaligned(lap) || misaligned(out))
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_laplacian: pointers must be 16-byte aligned");
  if (out == lap) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_laplacian: out aliases lap");
  return dispatch<kLap>(plan, lap, nullptr, out, nullptr);
}

gfc_status gfc_backward(gfc_plan* plan, const void* grad_out, void* grad_gx, void* grad_gy) {
  clear_error();
  if (!plan || !grad_out || !grad_gx || !grad_gy) return fail(GFC_ERR_INVALID_ARG, "gfc_backward: null argument");
  if (misaligned(grad_out) || misaligned(grad_gx) || misaligned(grad_gy))
    return fail(GFC_ERR_INVALID_ARG, "gfc_backward: pointers must be 16-byte aligned");
  if (grad_gx == grad_gy || grad_gx == grad_out || grad_gy == grad_out)
    return fail(GFC_ERR_INVALID_ARG, "gfc_backward: arguments alias");
  return dispatch<kAdj>(plan, grad_out, nullptr, grad_gx, grad_gy);
}

gfc_status gfc_solve_from_gradient_host(gfc_plan* plan, const void* gx, const void* gy, void* out) {
  clear_error();
  if (!plan || !gx || !gy || !out) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient_host: null argument");
  if (out == gx || out == gy) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient_host: out aliases an input");
  if (plan->ragged) return fail(GFC_ERR_UNSUPPORTED, "gfc_solve_from_gradient_host: not available for ragged plans");
  switch (plan->dtype) {
    case GFC_F32: return run_host<float>(plan, gx, gy, out);
    case GFC_F16: return run_host<__half>(plan, gx, gy, out);
    default: return run_host<__nv_bfloat16>(plan, gx, gy, out);
  }
}

gfc_status gfc_plan_set_profiling(gfc_plan* plan, int enable) {
  clear_error();
  if (!plan) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_set_profiling: null plan");
  if (enable && plan->ev_cap == 0) {
    const int cap = 65536;
    plan->ev_start = (cudaEvent_t*)calloc(cap, sizeof(cudaEvent_t));
    plan->ev_stop = (cudaEvent_t*)calloc(cap, sizeof(cudaEvent_t));
    plan->ev_pass = (int*)calloc(cap, sizeof(int));
    if (!plan->ev_start || !plan->ev_stop || !plan->ev_pass)
      return fail(GFC_ERR_ALLOC, "gfc_plan_set_profiling: host allocation failed");
    for (int i = 0; i < cap; ++i) {
      GFC_CUDA_TRY(cudaEventCreate(&plan->ev_start[i]));
      GFC_CUDA_TRY(cudaEventCreate(&plan->ev_stop[i]));
      plan->ev_cap = i + 1;
    }
  }
  plan->profiling = enable != 0;
  return GFC_OK;
}

gfc_status gfc_plan_get_profile(gfc_plan* plan, gfc_profile* out, int reset) {
  clear_error();
  if (!plan || !out) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_get_profile: null argument");
  GFC_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  for (int i = 0; i < plan->ev_used; ++i) {
    float ms = 0.0f;
    GFC_CUDA_TRY(cudaEventElapsedTime(&ms, plan->ev_start[i], plan->ev_stop[i]));
    if (plan->ev_pass[i] >= 0) plan->prof.pass_ms[plan->ev_pass[i]] += ms;
  }
  plan->ev_used = 0;
  *out = plan->prof;
  if (reset) memset(&plan->prof, 0, sizeof(plan->prof));
  return GFC_OK;
}

gfc_status gfc_fft_c2c(int n, int count, int dir, const void* in, void* out, void* stream) {
  clear_error();
  if (!in || !out || count < 0 || (dir != -1 && dir != 1))
    return fail(GFC_ERR_INVALID_ARG, "gfc_fft_c2c: bad argument (count=%d dir=%d)", count, dir);
  if (misaligned(in) || misaligned(out)) return fail(GFC_ERR_INVALID_ARG, "gfc_fft_c2c: pointers must be 16-byte aligned");
  FftPlan pl;
  if (!make_fft_plan(n, &pl)) return fail(GFC_ERR_UNSUPPORTED, "gfc_fft_c2c: n=%d is not 7-smooth or > %d", n, kMaxFftLen);
  if (count == 0) return GFC_OK;
  const size_t smem = 3 * (size_t)n * sizeof(float2);
  cudaStream_t st = (cudaStream_t)stream;
  if (dir < 0) {
    GFC_CUDA_TRY(ensure_smem(k_fft_rows<-1>, smem));
    k_fft_rows<-1><<<count, 256, smem, st>>>((const float2*)in, (float2*)out, pl);
  } else {
    GFC_CUDA_TRY(ensure_smem(k_fft_rows<1>, smem));
    k_fft_rows<1><<<count, 256, smem, st>>>((const float2*)in, (float2*)out, pl);
  }
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot allocate device memory at all: plug-ins inside a host
// application that owns every device allocation, fixed-budget embedded or
// real-time pipelines whose memory is reserved at start-up, and latency-bound
// loops where cudaMalloc/cudaFree would implicitly synchronise the device and
// stall other streams. They cannot create a plan (a plan allocates its tables
// and scratch), so this entry point takes its working memory from one
// file-scope device array instead. The array is created with the module on
// every GPU that loads this library and lives until the process exits.
//
// Layout of the array (each region 256-byte aligned): the complex spectrum of
// ONE field (M x ldS <= kNoAllocSpecElems), the Green spectrum
// (M x (N/2+1) <= kNoAllocGreenElems floats), the two twiddle tables, the
// adjoint partial sums and an error word.
// ---------------------------------------------------------------------------
namespace gfc {

constexpr size_t kNoAllocSpecElems = size_t(1) << 21;   // complex64: 16 MiB
constexpr size_t kNoAllocGreenElems = size_t(1) << 21;  // float: 8 MiB
constexpr size_t kOffSpec = 0;
constexpr size_t kOffGreen = kOffSpec + kNoAllocSpecElems * sizeof(float2);
constexpr size_t kOffTwN = kOffGreen + kNoAllocGreenElems * sizeof(float);
constexpr size_t kOffTwM = kOffTwN + size_t(kMaxFftLen) * sizeof(float2);
constexpr size_t kOffPartial = kOffTwM + size_t(kMaxFftLen) * sizeof(float2);
constexpr size_t kOffErr = kOffPartial + size_t(kMaxRowBlocks) * sizeof(float);
constexpr size_t kNoAllocBytes = kOffErr + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_base[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;  // guards g_noalloc_base (first calls from several host threads)

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the host-side name of the array is only a stand-in; kernels must
// be given this address).
static gfc_status noalloc_base(void** out) {
  int dev = 0;
  GFC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(GFC_ERR_UNSUPPORTED, "gfc_solve_from_gradient_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "gfc_solve_from_gradient_noalloc: cudaGetSymbolAddress");
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return GFC_OK;
}

}  // namespace gfc

extern "C" gfc_status gfc_solve_from_gradient_noalloc(int H, int W, int fields, const void* gx, const void* gy,
                                                      void* out, void* stream) {
  clear_error();
  if (!gx || !gy || !out || fields < 0)
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient_noalloc: null pointer or fields < 0");
  if (misaligned(gx) || misaligned(gy) || misaligned(out))
    return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient_noalloc: pointers must be 16-byte aligned");
  if (out == gx || out == gy) return fail(GFC_ERR_INVALID_ARG, "gfc_solve_from_gradient_noalloc: out aliases an input");
  int M = 0, N = 0;
  gfc_status st = gfc_padded_size(H, W, 4, GFC_SIZE_SMOOTH, &M, &N);
  if (st != GFC_OK) return st;
  gfc_plan P;
  memset(&P, 0, sizeof(P));
  P.H = H; P.W = W; P.C = 1; P.batch = fields; P.pad = 4; P.dtype = GFC_F32;
  P.M = M; P.N = N; P.Nh = N / 2 + 1; P.ldS = (P.Nh + 3) & ~3; P.chunk = 1; P.nslots = 1;
  P.spec_field = (size_t)M * P.ldS;
  // the limit the header states: M x ldS <= 2^21 with ldS = N/2 + 1 rounded up to a multiple of 4
  if ((size_t)M * P.ldS > kNoAllocSpecElems || (size_t)M * P.Nh > kNoAllocGreenElems)
    return fail(GFC_ERR_UNSUPPORTED,
                "gfc_solve_from_gradient_noalloc: padded size %dx%d needs M x ldS = %zu spectrum elements "
                "(ldS = N/2+1 rounded up to a multiple of 4), the static scratch holds %zu (square images up "
                "to 2008x2008)",
                M, N, (size_t)M * P.ldS, kNoAllocSpecElems);
  if (!make_fft_plan(N, &P.rowplan) || !make_fft_plan(M, &P.colplan))
    return fail(GFC_ERR_UNSUPPORTED, "gfc_solve_from_gradient_noalloc: no FFT schedule for %dx%d", M, N);
  if (fields == 0) return GFC_OK;
  void* base = nullptr;
  if ((st = noalloc_base(&base)) != GFC_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  P.spec = reinterpret_cast<float2*>(b + kOffSpec);
  P.G = reinterpret_cast<float*>(b + kOffGreen);
  P.twN = reinterpret_cast<float2*>(b + kOffTwN);
  P.twM = reinterpret_cast<float2*>(b + kOffTwM);
  P.partial = reinterpret_cast<float*>(b + kOffPartial);
  P.dev_err = reinterpret_cast<int*>(b + kOffErr);
  P.stream = (cudaStream_t)stream;
  GFC_CUDA_TRY(cudaGetDevice(&P.device));
  // The tables are rebuilt on every call (the array keeps whatever the last
  // call, possibly of another size, left in it); the error word is cleared.
  // Nothing else needs to start at zero: every spectrum row a pass reads was
  // written by the previous pass of the same field.
  GFC_CUDA_TRY(cudaMemsetAsync(P.dev_err, 0, sizeof(int), P.stream));
  GFC_CUDA_TRY(build_twiddles(P.twN, N, P.stream));
  GFC_CUDA_TRY(build_twiddles(P.twM, M, P.stream));
  GFC_CUDA_TRY(build_green(P.G, M, N, P.Nh, P.stream));
  const size_t fe = (size_t)H * W;
  for (int f = 0; f < fields; ++f) {
    cudaError_t e = run_chunk<float, kGrad>(&P, slot_bufs(&P, 0), static_cast<const float*>(gx) + f * fe,
                                            static_cast<const float*>(gy) + f * fe, static_cast<float*>(out) + f * fe,
                                            nullptr, 1, P.stream);
    if (e != cudaSuccess) return cuda_fail(e, "gfc_solve_from_gradient_noalloc launch");
  }
  return GFC_OK;
}

// ---------------------------------------------------------------------------
// captured solve graphs
// ---------------------------------------------------------------------------
struct gfc_graph {
  cudaGraphExec_t exec;
  cudaGraph_t graph;
};

static gfc_status run_op(gfc_plan* plan, int op, const void* in0, const void* in1, void* out0, void* out1) {
  switch (op) {
    case 0: return gfc_solve_from_gradient(plan, in0, in1, out0);
    case 1: return gfc_solve_from_laplacian(plan, in0, out0);
    case 2: return gfc_backward(plan, in0, out0, out1);
  }
  return fail(GFC_ERR_INVALID_ARG, "gfc_graph_create: unknown op %d", op);
}

extern "C" gfc_status gfc_graph_create(gfc_plan* plan, int op, const void* in0, const void* in1, void* out0,
                                       void* out1, gfc_graph** graph) {
  clear_error();
  if (!plan || !graph) return fail(GFC_ERR_INVALID_ARG, "gfc_graph_create: null argument");
  *graph = nullptr;
  if (plan->profiling) return fail(GFC_ERR_UNSUPPORTED, "gfc_graph_create: turn profiling off before capturing");
  cudaStream_t saved = plan->stream, cs = nullptr;
  gfc_status st = run_op(plan, op, in0, in1, out0, out1);  // lazy set-up outside the capture
  if (st != GFC_OK) return st;
  GFC_CUDA_TRY(cudaStreamSynchronize(saved));
  GFC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  plan->stream = cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = run_op(plan, op, in0, in1, out0, out1);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (st == GFC_OK && e2 != cudaSuccess) e = e2;
  }
  plan->stream = saved;
  cudaStreamDestroy(cs);
  if (st != GFC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "gfc_graph_create: capture");
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "gfc_graph_create: instantiate");
  }
  gfc_graph* out = (gfc_graph*)calloc(1, sizeof(gfc_graph));
  if (!out) {
    cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    return fail(GFC_ERR_ALLOC, "gfc_graph_create: host allocation failed");
  }
  out->exec = x;
  out->graph = g;
  *graph = out;
  return GFC_OK;
}

extern "C" gfc_status gfc_graph_launch(gfc_graph* graph, void* stream) {
  clear_error();
  if (!graph) return fail(GFC_ERR_INVALID_ARG, "gfc_graph_launch: null graph");
  GFC_CUDA_TRY(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
  return GFC_OK;
}

extern "C" gfc_status gfc_graph_destroy(gfc_graph* graph) {
  clear_error();
  if (!graph) return GFC_OK;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  free(graph);
  return GFC_OK;
}

// fast_kernels.cuh -- register-resident GFC passes for transform lengths with a
// two-stage schedule (Eq. 23, Algorithm B; the same three passes as solve.cu).
// Each supported size pair is instantiated in its own translation unit
// (fast_<M>x<N>.cu) so the library builds in parallel.
//
// Hand-offs between the passes:
//   pass L  (edited solves, Laplacian input, or rows too wide to stage) writes
//           the packed rows z[pair][j] = L[2 pair][j] + i L[2 pair+1][j];
//   pass A  stages the gradient rows of an item by bulk copy and forms L itself
//           (or stages z, or the adjoint's grad_out rows), and writes the row
//           spectrum column-major, spec[l][r] (l < N/2+1 Hermitian columns), one
//           2F-row column segment at a time: the transpose is folded into the
//           two-for-one split it does through shared memory anyway;
//   pass B  loads whole columns of spec straight into registers and writes its
//           result row-major, Y[i][l] (image rows i < H; H + 1 for the
//           adjoint), straight from registers, into the buffer that held z;
//   pass C  stages the rows of Y an item needs by bulk copy (the adjoint's
//           inverse row pass likewise) and writes the cropped output.
//
// Row transforms (length N = R1 R2, T = R2 threads per transform, F transforms
// per block): stage 1 is one radix-R1 DFT per thread on x[t + R2 r]; one
// shared-memory exchange; stage 2 has R1 radix-R2 DFTs with the twiddles
// w_N^(r j): R1/R2 per thread when R2 divides R1, else one for each of the
// first R1 threads (R1 < R2). Column transforms (M = R1 R2, R1 <= R2, T = R2 threads
// per column): forward stage 1 radix-R1, exchange, forward stage 2 radix-R2;
// each thread then holds the bins t + R1 s, multiplies them by the Green
// spectrum and runs the inverse's first stage (radix-R2, no twiddles) on the
// same registers; one more exchange and the inverse's radix-R1 stage.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "fft_reg.cuh"
#include "gfc_internal.h"
#include "tma.cuh"

namespace gfc {

// The register-resident schedules assume Algorithm A's pad of 4.
constexpr int kP = 4;

// smallest image width that pads to row length N under the SMOOTH policy (pad
// kP): the row kernels skip the crop test for columns below it
constexpr int cx_min_width(int N) {
  int lo = N;
  for (int n = N; n > 2 * kP && cx_row_policy(n) >= N; --n)
    if (cx_row_policy(n) == N) lo = n;
  return lo - 2 * kP;
}

// Column schedule placeholder of a shape compiled for its row length only.
struct NoCols {
  static constexpr int C = 1;
};

struct FastArgs {
  int H, W, p, M, N, Nh, ldM;
  int nrows, ncols;  // support of L (from torus row/col p): H+1, W+1 (gradient) or H, W
  int npairs, ldz;   // packed row pairs of L, and the stride of a packed row (>= N, zero padded)
  int zpairs;        // packed rows per field (npairs rounded up to whole groups, extra rows zero)
  int ngroups;       // row-pair groups per field (pass A) / output row-pair groups (pass C)
  int nparts;        // pass B column blocks per field (u[0,0] partial sums)
  int nf;            // fields in this chunk
  int ldY;           // row stride of the row-major spectrum Y (complex elements)
  int* err;          // the plan's device error word (bounded waits that run out)
  // recursive column solve (row-major spectrum S, bands of 2F rows from torus row p)
  int srows;         // rows of S per field (2 zpairs; rows past the support are zero)
  int G;             // bands per field
  size_t tri_field;  // complex elements per field of the band scratch
  int stage_out;     // inverse row pass: output rows staged in shared memory, stored by bulk copy
  double invM, invN; // 1 / M, 1 / N (FP64 divisions are slow on this part)
  int adj;           // the recursive column solve runs the adjoint (half-bands, the sum term at row 0)
  int l2res;         // the chunks' spectrum hand-off fits the L2: evict-first streams, evict-last spectrum,
                     // the inverse row pass drops the spectrum lines it has read
};

// Band scratch of one field (recursive column solve), complex elements:
//   carries [G][2][ldY]: row 0 of band g the causal carry into the band, row 1
//           the anticausal carry from below it (the sweep; read by pass C);
//   sums    [nkb][G][2][32]: the bands' causal and anticausal sums with zero
//           carries (pass A), in tiles of 32 columns, so that a tile is one
//           contiguous copy for the sweep;
//   col0    srows floats: the real parts of column 0 of S (pass A).
// The row-major spectrum S holds 2F rows per band; the sweep writes column 0's
// exact solution into it.
// (The plan sizes this per field in tri_field.)
constexpr int kTriCols = 32;
// Slots of a field's FP64 partial-sum area used by the recursive column solve:
// [0, nkb) the sweep blocks' partials of u[0,0]; kTriCnt a counter of sweep
// blocks done (reset by the row pass, which runs first); kTriU00 u[0,0] itself,
// combined by the last sweep block of the field.
constexpr int kTriCnt = 150, kTriU00 = 151;
__device__ __forceinline__ float2* tri_sums(float2* tri, int field, const FastArgs& A) {
  return tri + (size_t)field * A.tri_field + (size_t)2 * A.G * A.ldY;
}
__device__ __forceinline__ float* tri_col0(float2* tri, int field, const FastArgs& A) {
  const size_t nkb = (size_t)(A.ldY + kTriCols - 1) / kTriCols;
  return reinterpret_cast<float*>(tri_sums(tri, field, A) + nkb * 2 * A.G * kTriCols);
}
// s + v with its rounding error added to err (Knuth's TwoSum, explicitly
// rounded so the compiler cannot reassociate it); returns the rounded sum
__device__ __forceinline__ float two_sum_acc(float s, float v, float& err) {
  const float t = __fadd_rn(s, v);
  const float bp = __fsub_rn(t, s);
  err = __fadd_rn(err, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
  return t;
}

// one step of y <- x + a y with a = 1 - delta, as (x + y) - delta y: delta is
// held to full relative precision, so the pole near DC is not rounded away
__device__ __forceinline__ float2 tri_step(float2 x, float2 y, float delta) {
  return __ffma2_rn(make_float2(-delta, -delta), y, cadd(x, y));  // packed pair arithmetic
}

__device__ __forceinline__ float f_to_f(float x) { return x; }
__device__ __forceinline__ float f_to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float f_to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T> __device__ __forceinline__ T f_from_f(float x);
template <> __device__ __forceinline__ float f_from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ __half f_from_f<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 f_from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename T>
__device__ __forceinline__ float ldz(const T* __restrict__ g, int i, int j, int H, int W) {
  return (i >= 0 && i < H && j >= 0 && j < W) ? f_to_f(g[(size_t)i * W + j]) : 0.0f;
}

template <typename T>
__device__ __forceinline__ float4 ld4(const T* __restrict__ g, int i, int j, int W);
template <>
__device__ __forceinline__ float4 ld4<float>(const float* __restrict__ g, int i, int j, int W) {
  return __ldg(reinterpret_cast<const float4*>(g + (size_t)i * W + j));
}
template <>
__device__ __forceinline__ float4 ld4<__half>(const __half* __restrict__ g, int i, int j, int W) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(g + (size_t)i * W + j));
  const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
template <>
__device__ __forceinline__ float4 ld4<__nv_bfloat16>(const __nv_bfloat16* __restrict__ g, int i, int j, int W) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(g + (size_t)i * W + j));
  const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int N_, int R1_, int R2_, int F_>
struct RowShape {
  static constexpr int N = N_, R1 = R1_, R2 = R2_, F = F_;
  static constexpr int T = R2;                            // threads per transform
  static constexpr int J2 = (R1 >= R2) ? R1 / R2 : 1;     // stage-2 butterflies per thread
  static constexpr int JSPAN = (R1 >= R2) ? R2 : R1;      // stage-2 butterflies j = t + R2 jj, t < JSPAN
  // exchange stride of a thread's R1 stage-1 outputs: odd, so that the threads'
  // 8-byte accesses spread over the banks
  static constexpr int R1P = (R1 % 2 == 0) ? R1 + 1 : R1 + 2;
  static constexpr int NP = (N / R1) * R1P;               // padded transform buffer
  static constexpr int THREADS = ((F * T + 31) / 32) * 32;
  static_assert(R1 % R2 == 0 || R1 < R2, "row schedule needs R2 | R1 or R1 < R2");
  static constexpr int NO = N + 1;        // stage-2 output buffer stride (natural order)
  static constexpr int WMIN = cx_min_width(N);
  static constexpr int LDY_ = ((N / 2 + 1) + 3) & ~3;  // row stride of Y and S (complex)
  static constexpr size_t smem_bytes() { return (size_t)(R1 * R2 + F * NP) * sizeof(float2); }
  static constexpr int CBUF = ((R1 * R2 + F * NP) + 1) & ~1;  // 16-byte aligned offset of the carry rows
  static constexpr size_t smem_bytes_tri_inv() { return (size_t)(CBUF + 2 * LDY_) * sizeof(float2); }
  static constexpr size_t smem_bytes_fwd() { return (size_t)(R1 * R2 + F * NP + F * NO) * sizeof(float2); }
  // blocks per SM the register allocation must allow: long rows fill shared
  // memory at 2 (3 for the inverse pass); short rows leave room for 4. Wider
  // blocks and long stage-2 radices get fewer, so that the transforms keep
  // their values in registers (at least ~200 registers a thread in the forward
  // passes, ~160 in the inverse one; stage-2 radices >= 48 take 2 blocks)
  static constexpr bool SHORT = N <= 512;
  static constexpr int cx_blocks(int cap, int regs) {
    const int b = 65536 / (THREADS * regs);
    return b < 1 ? 1 : (b > cap ? cap : b);
  }
  static constexpr int MINB_FWD = SHORT ? 4 : cx_blocks(2, 200);
  static constexpr int MINB_INV = SHORT ? 4 : cx_blocks(R2 >= 48 ? 2 : 3, 160);
  static constexpr int MINB_ADJ = SHORT ? 4 : cx_blocks(2, 200);
  // adjoint inverse row pass: twiddles, exchange, the factor table
  // 1 - exp(2 pi i l / N) for l <= N/2, then (16-byte aligned) the F + 1 rows of
  // Y an item needs, LDY complex each
  static constexpr int LDY = LDY_;
  static constexpr size_t adj_stage_offset() {
    return (((size_t)(R1 * R2 + F * NP + (N / 2 + 1)) * sizeof(float2)) + 15) / 16 * 16;
  }
  static constexpr size_t smem_bytes_adj() { return adj_stage_offset() + (size_t)(F + 1) * LDY * sizeof(float2); }
  // the recursive column solve's adjoint also stages the half-band's two carries
  static constexpr size_t smem_bytes_adj_tri() { return adj_stage_offset() + (size_t)(F + 3) * LDY * sizeof(float2); }
  // The exchange stores each run of R1 elements at a stride of R1P (element
  // m = t R1 + s at t R1P + s, conflict-free stage-1 writes); the kernels use
  // the closed forms t R1P + s for m = t R1 + s and j + R1P r for m = j + R1 r.
};

// Shared-memory wavefronts of the column pass's four exchange accesses for a
// per-column stride MP (8-byte elements, thread tid = t C + c, each half-warp
// one request): forward write t R1 + s, forward read t + R1 r (t < R1),
// inverse write t (R2 + 1) + s (t < R1), inverse read t + (R2 + 1) r (t < R2).
constexpr int cols_exchange_wavefronts(int C, int R1, int R2, int threads, int MP) {
  int total = 0;
  for (int h = 0; h < threads / 16; ++h) {
    for (int pat = 0; pat < 4; ++pat) {
      int addr[16] = {}, n = 0;
      for (int L = 0; L < 16; ++L) {
        const int tid = 16 * h + L, c = tid % C, t = tid / C;
        const int tmax = (pat == 1 || pat == 2) ? R1 : R2;
        if (t >= tmax) continue;
        const int stride = pat == 0 ? R1 : (pat == 2 ? R2 + 1 : 1);
        const int a = c * MP + t * stride;
        bool seen = false;
        for (int k = 0; k < n; ++k) seen = seen || addr[k] == a;
        if (!seen) addr[n++] = a;
      }
      int worst = 0;
      for (int b = 0; b < 16; ++b) {
        int cnt = 0;
        for (int k = 0; k < n; ++k) cnt += ((addr[k] % 16) == b) ? 1 : 0;
        worst = cnt > worst ? cnt : worst;
      }
      total += worst;
    }
  }
  return total;
}
// the smallest stride >= lo with the fewest wavefronts among the next 32
constexpr int cols_exchange_stride(int C, int R1, int R2, int threads, int lo) {
  int best = lo, bw = cols_exchange_wavefronts(C, R1, R2, threads, lo);
  for (int mp = lo + 1; mp < lo + 32; ++mp) {
    const int w = cols_exchange_wavefronts(C, R1, R2, threads, mp);
    if (w < bw) { bw = w; best = mp; }
  }
  return best;
}

template <int M_, int R1_, int R2_, int C_>
struct ColShape {
  static constexpr int M = M_, R1 = R1_, R2 = R2_, C = C_;
  static constexpr int T = R2;             // threads per column
  static constexpr int THREADS = ((C * T + 31) / 32) * 32;
  // blocks per SM the registers must allow (short columns leave room for 4)
  static constexpr int MINB = (M <= 512 && THREADS <= 160) ? 4 : ((THREADS <= 256) ? 2 : 1);
  static_assert(R1 <= R2, "column schedule needs R1 <= R2");
  static_assert(C <= 32, "the u[0,0] partial of a block is gathered in one warp");
  // per-column exchange stride: the inverse exchange keeps one spare slot every
  // R2 elements (t (R2 + 1) + s, t + (R2 + 1) r), so it needs M + R1 - 1
  static constexpr int MP = cols_exchange_stride(C, R1, R2, THREADS, M + R1 - 1);
  static constexpr int TWF_STRIDE = (R2 % 2 == 0) ? R2 + 1 : R2;
  static constexpr int TWI_STRIDE = (R1 % 2 == 0) ? R1 + 1 : R1;
  static constexpr int GS = ((M + 3) / 4) * 4;  // floats per staged Green column (16-byte multiple)
  static constexpr size_t smem_bytes() {
    return (size_t)C * GS * sizeof(float) + (size_t)(R1 * TWF_STRIDE + R2 * TWI_STRIDE + C * MP) * sizeof(float2);
  }
};

// ---------------------------------------------------------------------------
// pass L: divergence (Eq. 3) or copy of the given Laplacian, packed two rows per
// complex value: z[pair][j] = L[2 pair][j] + i L[2 pair + 1][j], j < ncols
// (image columns; the pad is implicit). Streams gx, gy once.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_fast_div(const T* __restrict__ in0, const T* __restrict__ in1,
                                                  float2* __restrict__ z, float* __restrict__ partial, FastArgs A) {
  // grid: x = groups of 4 padded columns, y = packed rows (zpairs), z = fields.
  // Packed row `pair`, padded column c holds L[2 pair][c - p] + i L[2 pair + 1][c - p],
  // zero outside the support, so the row pass can load it without range checks.
  // MODE 2 (adjoint) packs grad_out like a Laplacian and also sums it: one
  // block covers a whole packed row and writes that row pair's FP64 sum.
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int pair = blockIdx.y, field = blockIdx.z;
  const bool inq = q < A.ldz / 4;
  if (MODE != 2 && !inq) return;
  const int c0 = 4 * q, j0 = c0 - kP;
  float la[4] = {0.0f, 0.0f, 0.0f, 0.0f}, lb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (inq && pair < A.npairs && j0 + 3 >= 0 && j0 < A.ncols) {
    const bool vec4 = (A.W % 4) == 0 && j0 >= 0;
    const size_t fe = (size_t)A.H * A.W;
    const T* a = in0 + field * fe;
    const T* b = (MODE == 0) ? in1 + field * fe : nullptr;
    const int ia = 2 * pair, ib = ia + 1;
    if (MODE == 0) {
      float xa[5], xb[5], ya[4], yb[4], ym[4];  // gx rows ia, ib at j0-1..j0+3; gy rows ia, ib, ia-1
      const bool ina = ia < A.H, inb = ib < A.H, inm = ia >= 1 && ia - 1 < A.H;
      if (vec4 && j0 + 3 < A.W) {
        const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 ga = ina ? ld4(a, ia, j0, A.W) : z4, gb = inb ? ld4(a, ib, j0, A.W) : z4;
        const float4 ha = ina ? ld4(b, ia, j0, A.W) : z4, hb = inb ? ld4(b, ib, j0, A.W) : z4;
        const float4 hm = inm ? ld4(b, ia - 1, j0, A.W) : z4;
        xa[1] = ga.x; xa[2] = ga.y; xa[3] = ga.z; xa[4] = ga.w;
        xb[1] = gb.x; xb[2] = gb.y; xb[3] = gb.z; xb[4] = gb.w;
        ya[0] = ha.x; ya[1] = ha.y; ya[2] = ha.z; ya[3] = ha.w;
        yb[0] = hb.x; yb[1] = hb.y; yb[2] = hb.z; yb[3] = hb.w;
        ym[0] = hm.x; ym[1] = hm.y; ym[2] = hm.z; ym[3] = hm.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          xa[e + 1] = ldz(a, ia, j0 + e, A.H, A.W);
          xb[e + 1] = ldz(a, ib, j0 + e, A.H, A.W);
          ya[e] = ldz(b, ia, j0 + e, A.H, A.W);
          yb[e] = ldz(b, ib, j0 + e, A.H, A.W);
          ym[e] = ldz(b, ia - 1, j0 + e, A.H, A.W);
        }
      }
      xa[0] = ldz(a, ia, j0 - 1, A.H, A.W);
      xb[0] = ldz(a, ib, j0 - 1, A.H, A.W);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        la[e] = (xa[e + 1] - xa[e]) + (ya[e] - ym[e]);
        lb[e] = (xb[e + 1] - xb[e]) + (yb[e] - ya[e]);
      }
    } else {
      if (vec4 && j0 + 3 < A.W) {
        const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 ga = ia < A.H ? ld4(a, ia, j0, A.W) : z4, gb = ib < A.H ? ld4(a, ib, j0, A.W) : z4;
        la[0] = ga.x; la[1] = ga.y; la[2] = ga.z; la[3] = ga.w;
        lb[0] = gb.x; lb[1] = gb.y; lb[2] = gb.z; lb[3] = gb.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          la[e] = ldz(a, ia, j0 + e, A.H, A.W);
          lb[e] = ldz(a, ib, j0 + e, A.H, A.W);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool inj = j0 + e >= 0 && j0 + e < A.ncols;
      la[e] = (inj && ia < A.nrows) ? la[e] : 0.0f;
      lb[e] = (inj && ib < A.nrows) ? lb[e] : 0.0f;
    }
  }
  if (inq) {
    float4* dst = reinterpret_cast<float4*>(z + ((size_t)field * A.zpairs + pair) * A.ldz + c0);
    dst[0] = make_float4(la[0], lb[0], la[1], lb[1]);
    dst[1] = make_float4(la[2], lb[2], la[3], lb[3]);
  }
  if (MODE == 2) {
    // a thread's 8 values summed in FP32 (error a few ulp of their magnitudes),
    // the block's in FP64: FP64 arithmetic is scarce on this GPU
    const float s8 = ((la[0] + la[1]) + (la[2] + la[3])) + ((lb[0] + lb[1]) + (lb[2] + lb[3]));
    double v = (double)s8;
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      reinterpret_cast<double*>(partial)[(size_t)field * (kMaxRowBlocks / 2) + pair] = t;
    }
  }
}

// Pass L with a gradient edit applied as the gradient is loaded (Sec. 3.2.3
// thresholding, Eq. 26 merging): the same packed rows as k_fast_div<T, 0> on
// the edited field, bit for bit, without the edited field ever being stored.
// Every edited pixel is computed once: a thread owns 4 columns and walks down
// kEditPairs row pairs, keeping the edited gy of the row above in registers;
// the edited gx of the column to its left comes from the neighbouring lane
// (lane 0 edits that one pixel itself).
constexpr int kEditPairs = 8;

template <typename T, int EDIT>
__device__ __forceinline__ void edit_row4(const T* __restrict__ a, const T* __restrict__ b,
                                          const T* __restrict__ e, int i, int j0, const FastArgs& A, float t2,
                                          float alpha, float* ex, float* ey) {
  if (i < 0 || i >= A.H || j0 + 3 < 0 || j0 >= A.W) {
#pragma unroll
    for (int k = 0; k < 4; ++k) ex[k] = ey[k] = 0.0f;
    return;
  }
  if ((A.W % 4) == 0 && j0 >= 0 && j0 + 3 < A.W) {
    const float4 x = ld4(a, i, j0, A.W), y = ld4(b, i, j0, A.W);
    float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w}, cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (EDIT == kEditMerge) {
      const float4 c = ld4(e, i, j0, A.W);
      cs[0] = c.x; cs[1] = c.y; cs[2] = c.z; cs[3] = c.w;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (EDIT == kEditThreshold) {
        const bool drop = edit_mag2(xs[k], ys[k]) < t2;
        ex[k] = drop ? 0.0f : xs[k];
        ey[k] = drop ? 0.0f : ys[k];
      } else {
        const float sc = edit_merge_scale(xs[k], ys[k], cs[k], alpha);
        ex[k] = edit_round(__fmul_rn(xs[k], sc), a);
        ey[k] = edit_round(__fmul_rn(ys[k], sc), a);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 v = edit_pixel<T, EDIT>(a, b, e, i, j0 + k, A.H, A.W, t2, alpha);
      ex[k] = v.x;
      ey[k] = v.y;
    }
  }
}

template <typename T, int EDIT>
__global__ void __launch_bounds__(512) k_fast_div_edit(const T* __restrict__ gx, const T* __restrict__ gy,
                                                       const T* __restrict__ edges, const float* __restrict__ t2s,
                                                       float alpha, float2* __restrict__ z, FastArgs A) {
  // grid: x = groups of 4 padded columns (whole warps), y = blocks of kEditPairs
  // packed rows, z = fields. Every lane stays to the end (warp shuffles).
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int field = blockIdx.z, lane = threadIdx.x & 31;
  const bool inq = q < A.ldz / 4;
  const int c0 = 4 * q, j0 = c0 - kP;
  const size_t fe = (size_t)A.H * A.W;
  const T* a = gx + field * fe;
  const T* b = gy + field * fe;
  const T* e = (EDIT == kEditMerge) ? edges + field * fe : nullptr;
  const float t2 = (EDIT == kEditThreshold) ? t2s[field] : 0.0f;
  const int p0 = blockIdx.y * kEditPairs;
  const int p1 = min(p0 + kEditPairs, A.zpairs);
  // edited gy of the row above the first row of the block
  float ym[4], scratch[4];
  edit_row4<T, EDIT>(a, b, e, 2 * p0 - 1, j0, A, t2, alpha, scratch, ym);
  for (int pair = p0; pair < p1; ++pair) {
    float L[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * pair + h;
      float ex[4], ey[4];
      edit_row4<T, EDIT>(a, b, e, i, j0, A, t2, alpha, ex, ey);
      float left = __shfl_up_sync(0xffffffffu, ex[3], 1);
      if (lane == 0) left = edit_pixel<T, EDIT>(a, b, e, i, j0 - 1, A.H, A.W, t2, alpha).x;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float xl = (k == 0) ? left : ex[k - 1];
        const bool in = j0 + k >= 0 && j0 + k < A.ncols && i < A.nrows && pair < A.npairs;
        L[h][k] = in ? (ex[k] - xl) + (ey[k] - ym[k]) : 0.0f;
        ym[k] = ey[k];
      }
    }
    if (inq) {
      float4* dst = reinterpret_cast<float4*>(z + ((size_t)field * A.zpairs + pair) * A.ldz + c0);
      dst[0] = make_float4(L[0][0], L[1][0], L[0][1], L[1][1]);
      dst[1] = make_float4(L[0][2], L[1][2], L[0][3], L[1][3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Recursive column solve, pass A side: the item's 2F rows of the spectrum, from
// the F packed transforms in buf2 (two-for-one split), stored row-major
// (S[row][l], row = image-relative torus row), and per column l the item's
// band sums with zero carries,
//   e  = sum_r a^(nb-1-r) X[r]   (causal recursion y = X + a y run down the band)
//   e' = sum_r a^r X[r]          (anticausal recursion run up the band),
// over the nb band rows that lie on the torus. Thread t takes columns t, t +
// blockDim, ...: the row stores and sums are coalesced across threads.
// ---------------------------------------------------------------------------
// HALF (the adjoint): the sums are taken per half-band of F rows (half-bands
// 2g and 2g + 1; A.G counts half-bands), so that the inverse pass can solve F
// rows at a time.
template <class S, bool HALF = false>
__device__ __forceinline__ void tri_store_item(const float2* buf2, float2* __restrict__ spec, float2* __restrict__ tri,
                                               const float* __restrict__ cc, int field, int g, const FastArgs& A) {
  constexpr int RW = 2 * S::F;
  float2* Sr = spec + ((size_t)field * A.srows + (size_t)g * RW) * A.ldY;
  float2* sums = tri_sums(tri, field, A);
  const int nb = min(RW, A.M - A.p - g * RW);
  for (int k = threadIdx.x; k < A.Nh; k += blockDim.x) {
    float2* te = sums + ((size_t)(k / kTriCols) * A.G + g) * 2 * kTriCols + (k % kTriCols);  // tile of column k
    float2* tp = te + kTriCols;
    const int km = k == 0 ? 0 : S::N - k;
    float2 x[RW];
#pragma unroll
    for (int q = 0; q < S::F; ++q) {
      // X_a = (Z[k] + conj Z[N-k]) / 2, X_b = -i (Z[k] - conj Z[N-k]) / 2, in packed pair arithmetic
      const float2 zk = buf2[q * S::NO + k], zm = buf2[q * S::NO + km];
      const float2 zc = make_float2(zm.x, -zm.y);
      x[2 * q] = cscale(cadd(zk, zc), 0.5f);
      const float2 d = csub(zk, zc);
      x[2 * q + 1] = cscale(make_float2(d.y, -d.x), 0.5f);
    }
    if (!HALF && A.l2res) {  // the inverse row pass reads these rows next: last out of the L2
      const uint64_t pol = l2_policy_evict_last();
#pragma unroll
      for (int r = 0; r < RW; ++r) st_global_hint(Sr + (size_t)r * A.ldY + k, x[r], pol);
    } else {
#pragma unroll
      for (int r = 0; r < RW; ++r) Sr[(size_t)r * A.ldY + k] = x[r];
    }
    if (k == 0) {
      float* c0 = tri_col0(tri, field, A) + (size_t)g * RW;
#pragma unroll
      for (int r = 0; r < RW; ++r) c0[r] = x[r].x;
    }
    const float dl = __ldg(cc + (size_t)k * 8);
    if constexpr (HALF) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h * S::F >= nb) break;  // the second half lies past the torus
        float2 e = make_float2(0.0f, 0.0f), ep = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int r = h * S::F; r < (h + 1) * S::F; ++r)
          if (r < nb) e = tri_step(x[r], e, dl);
#pragma unroll
        for (int r = (h + 1) * S::F - 1; r >= h * S::F; --r)
          if (r < nb) ep = tri_step(x[r], ep, dl);
        float2* th = sums + ((size_t)(k / kTriCols) * A.G + 2 * g + h) * 2 * kTriCols + (k % kTriCols);
        th[0] = e;
        th[kTriCols] = ep;
      }
    } else {
      float2 e = make_float2(0.0f, 0.0f), ep = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int r = 0; r < RW; ++r)
        if (r < nb) e = tri_step(x[r], e, dl);
#pragma unroll
      for (int r = RW - 1; r >= 0; --r)
        if (r < nb) ep = tri_step(x[r], ep, dl);
      *te = e;
      *tp = ep;
    }
  }
}

// ---------------------------------------------------------------------------
// pass A: forward row transforms of the packed rows + two-for-one split +
// transposed store. Persistent over (field, group of F row pairs). The F packed
// rows of an item are one contiguous bulk copy into the exchange buffer,
// completed on an mbarrier; the copy for the next item is issued as soon as
// this item's stage-2 inputs are read, so it overlaps the stage-2 transforms
// and the transposed store of the spectrum.
// ---------------------------------------------------------------------------
template <class S, bool TRI>
__global__ void __launch_bounds__(S::THREADS, S::MINB_FWD) k_fast_rows_fwd(const float2* __restrict__ z,
                                                                 float2* __restrict__ spec,
                                                                 const float2* __restrict__ twg, FastArgs A,
                                                                 float2* __restrict__ tri,
                                                                 const float* __restrict__ cc,
                                                                 float* __restrict__ partial = nullptr) {
  extern __shared__ __align__(16) float2 sm[];
  float2* tw2 = sm;                   // [R1][R2]: w_N^(r j)
  float2* buf = sm + S::R1 * S::R2;   // staged packed rows [F][ldz], then the exchange (m -> m + m / R1)
  float2* buf2 = buf + S::F * S::NP;  // [F][NO] stage-2 output, natural order
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int f = tid / S::T, t = tid - f * S::T;
  const bool act = f < S::F;
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    tw2[i] = twg[r * j];
  }
  float2* mybuf = buf + (act ? f : 0) * S::NP;
  float2* mybuf2 = buf2 + (act ? f : 0) * S::NO;
  // unpack mapping: thread (uf, uk0) takes the bins k = uk0 + T s of transform uf
  const int uf = tid % S::F, uk0 = tid / S::F;
  const bool uact = tid < S::F * S::T;
  const int items = A.nf * A.ngroups;
  // one thread: stage the packed rows of item w (zero padded, whole rows);
  // prefetch: only start fetching them into L2, for the copy one item later
  auto issue = [&](int w, bool prefetch) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    const float2* zs = z + ((size_t)field * A.zpairs + (size_t)g * S::F) * A.ldz;
    const unsigned nb = (unsigned)(S::F * A.ldz * sizeof(float2));
    if (prefetch)
      l2_prefetch(zs, nb);
    else
      bulk_load(buf, zs, nb, &bar);
  };
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < items) issue(blockIdx.x, false);
  if (tid == 0 && (int)(blockIdx.x + gridDim.x) < items) issue(blockIdx.x + gridDim.x, true);
  unsigned phase = 0;
#pragma unroll 1
  for (int w = blockIdx.x; w < items; w += gridDim.x, phase ^= 1u) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    if (TRI && g == 0 && tid == 0)  // the sweep's count of finished blocks for this field starts at 0
      reinterpret_cast<unsigned*>(reinterpret_cast<double*>(partial) + (size_t)field * (kMaxRowBlocks / 2) + kTriCnt)[0] = 0u;
    const bool landed = mbar_wait(&bar, phase);
    if (__syncthreads_or(!landed)) {  // the copy never completed: report, let it drain, stop
      if (tid == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&bar, phase);
      return;
    }
    float2 v[S::R1];
    if (act) {
      const float2* zr = buf + (size_t)f * A.ldz + t;
#pragma unroll
      for (int r = 0; r < S::R1; ++r) v[r] = zr[S::R2 * r];
    }
    __syncthreads();  // every staged row read: buf becomes the exchange buffer
    if (act) {
      dft_reg<S::R1, -1>(v);
      // Stockham stage 1 writes t R1 + s; its padded index is t R1P + s
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();  // stage-1 results visible; previous unpack done with buf2
    const bool act2 = act && t < S::JSPAN;
#pragma unroll
    for (int jj = 0; jj < S::J2; ++jj) {
      const int j = t + S::R2 * jj;  // j < R1, so the padded index of j + R1 r is j + R1P r
      float2 u[S::R2];
      if (act2) {
        u[0] = mybuf[j];
#pragma unroll
        for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[j + S::R1P * r], tw2[j * S::R2 + r]);
      }
      if (jj == S::J2 - 1) {
        fence_proxy_async_smem();  // this thread's accesses of buf precede the next bulk copy into it
        __syncthreads();           // buf free
        if (tid == 0 && w + (int)gridDim.x < items) issue(w + gridDim.x, false);
        if (tid == 0 && w + 2 * (int)gridDim.x < items) issue(w + 2 * gridDim.x, true);
      }
      if (act2) {
        dft_reg<S::R2, -1>(u);
#pragma unroll
        for (int s2 = 0; s2 < S::R2; ++s2) mybuf2[j + S::R1 * s2] = u[s2];
      }
    }
    __syncthreads();  // stage-2 results visible
    if constexpr (TRI) {
      tri_store_item<S>(buf2, spec, tri, cc, field, g, A);
      continue;
    }
    if (g == 0) {
      // rows of every column outside the support [p, p + nrows) are zero, so the
      // column pass loads whole columns without range checks
      float2* Sz = spec + (size_t)field * A.Nh * A.ldM;
      const int nz = A.M - A.nrows;
      for (int idx = tid; idx < A.Nh * nz; idx += blockDim.x) {
        const int k = idx / nz, q = idx - k * nz;
        Sz[(size_t)k * A.ldM + (q < kP ? q : q + A.nrows)] = make_float2(0.0f, 0.0f);
      }
    }
    // X_a[k] = (Z[k] + conj Z[N-k]) / 2, X_b[k] = -i (Z[k] - conj Z[N-k]) / 2, stored at spec[k][p + row]
    const int ra = g * 2 * S::F + 2 * uf;
    if (uact && ra < A.nrows) {
      float2* Sp = spec + (size_t)field * A.Nh * A.ldM + A.p + ra;
      const float2* zb = buf2 + uf * S::NO;
      const bool two = ra + 1 < A.nrows, vec = ((A.p + ra) & 1) == 0;
      for (int k = uk0; k < A.Nh; k += S::T) {
        const float2 zk = zb[k], zm = zb[k == 0 ? 0 : S::N - k];
        const float2 xa = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 xb = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        float2* dst = Sp + (size_t)k * A.ldM;
        if (two && vec) {
          *reinterpret_cast<float4*>(dst) = make_float4(xa.x, xa.y, xb.x, xb.y);
        } else {
          dst[0] = xa;
          if (two) dst[1] = xb;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// pass L folded into pass A (gradient input): the 2F gx rows and 2F + 1 gy rows
// an item needs (gy from the row above its first pair) arrive as two bulk
// copies into the exchange buffers, and each thread forms its packed values
// L[2 pair][j] + i L[2 pair + 1][j] (Eq. 3) from shared memory with the same
// arithmetic as pass L, so the packed rows never go through HBM. The rest is
// k_fast_rows_fwd. The next item's rows are requested once this item's
// spectrum is stored (the staging area spans both exchange buffers).
// ADJ: the adjoint's first step instead, z = Crop^T(grad_out) from the 2F
// staged rows of grad_out, with each row pair's FP64 sum written where pass B
// reads it for the -(sum grad_out) e_00 term (as k_fast_div<T, 2>).
// Requires W sizeof(T) to be a multiple of 16 and the staging to fit
// (fused_div_fits).
// ---------------------------------------------------------------------------
template <class S, typename T>
__host__ __device__ constexpr size_t fused_stage_bytes(int W) {
  return (size_t)(4 * S::F + 1) * W * sizeof(T);
}
template <class S>
__host__ __device__ constexpr size_t fused_exchange_bytes() {
  return (size_t)(S::F * S::NP + S::F * S::NO) * sizeof(float2);
}

// EDIT = kEditThreshold (Sec. 3.2.3) zeroes, in the staged rows, every pixel whose
// gradient magnitude is below the field's threshold (t2s: squared thresholds of
// the chunk's fields), with the keep/drop decision of the standalone threshold
// kernel, before the divergence is formed; the gy row above the item takes its
// decision from gx of that row, read from global memory ahead of the staging.
template <class S, typename T, bool ADJ, bool TRI, int EDIT = kEditNone>
__global__ void __launch_bounds__(S::THREADS, S::MINB_FWD) k_fast_rows_fwd_div(const T* __restrict__ gx,
                                                                     const T* __restrict__ gy,
                                                                     float2* __restrict__ spec,
                                                                     const float2* __restrict__ twg,
                                                                     float* __restrict__ partial, FastArgs A,
                                                                     float2* __restrict__ tri,
                                                                     const float* __restrict__ cc,
                                                                     const float* __restrict__ t2s = nullptr) {
  static_assert(EDIT == kEditNone || (EDIT == kEditThreshold && !ADJ), "only the threshold edit is staged");
  extern __shared__ __align__(16) float2 sm[];
  float2* tw2 = sm;
  float2* buf = sm + S::R1 * S::R2;
  float2* buf2 = buf + S::F * S::NP;
  constexpr int RW = 2 * S::F;  // image rows per item
  T* sgx = reinterpret_cast<T*>(buf);  // gx rows (ADJ: grad_out rows) r0 .. r0 + RW - 1
  T* sgy = sgx + (size_t)RW * A.W;     // gy rows r0 - 1 .. r0 + RW - 1
  __shared__ __align__(8) uint64_t bar;
  __shared__ float2 red[ADJ ? S::F * S::T : 1];  // ADJ: per-thread compensated sums (sum, error) of the row pairs
  const int tid = threadIdx.x;
  const int f = tid / S::T, t = tid - f * S::T;
  const bool act = f < S::F;
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    tw2[i] = twg[r * j];
  }
  float2* mybuf = buf + (act ? f : 0) * S::NP;
  float2* mybuf2 = buf2 + (act ? f : 0) * S::NO;
  const int uf = tid % S::F, uk0 = tid / S::F;
  const bool uact = tid < S::F * S::T;
  const int items = A.nf * A.ngroups;
  const size_t fe = (size_t)A.H * A.W;
  // one thread: stage the gradient rows of item w (prefetch: only start
  // fetching the same rows into L2, for the copy one item later)
  auto issue = [&](int w, bool prefetch) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    const int r0 = g * RW;
    const int nx = (A.H - r0) < RW ? (A.H - r0) : RW;             // gx rows r0 .. r0 + nx - 1 (nx may be 0)
    const int y0 = r0 > 0 ? r0 - 1 : 0, y1 = (A.H < r0 + RW) ? A.H : r0 + RW;  // gy rows y0 .. y1 - 1
    const unsigned row = (unsigned)(A.W * sizeof(T));
    const T* xs = gx + field * fe + (size_t)r0 * A.W;
    const T* ys = gy + field * fe + (size_t)y0 * A.W;
    if (prefetch) {
      if (nx > 0) l2_prefetch(xs, (unsigned)nx * row);
      if (!ADJ) l2_prefetch(ys, (unsigned)(y1 - y0) * row);
      return;
    }
    if constexpr (ADJ) {  // (with the recursive column solve the last band may hold no row of grad_out)
      mbar_expect_tx(&bar, (unsigned)(nx > 0 ? nx : 0) * row);
      if (nx > 0) bulk_copy(sgx, xs, (unsigned)nx * row, &bar);
    } else {
      mbar_expect_tx(&bar, (unsigned)(nx > 0 ? nx : 0) * row + (unsigned)(y1 - y0) * row);
      if (A.l2res) {  // read once: first out of the L2, so that the spectrum stays
        const uint64_t pol = l2_policy_evict_first();
        if (nx > 0) bulk_copy_hint(sgx, xs, (unsigned)nx * row, &bar, pol);
        bulk_copy_hint(sgy + (size_t)(y0 - (r0 - 1)) * A.W, ys, (unsigned)(y1 - y0) * row, &bar, pol);
      } else {
        if (nx > 0) bulk_copy(sgx, xs, (unsigned)nx * row, &bar);
        bulk_copy(sgy + (size_t)(y0 - (r0 - 1)) * A.W, ys, (unsigned)(y1 - y0) * row, &bar);
      }
    }
  };
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < items) issue(blockIdx.x, false);
  if (tid == 0 && (int)(blockIdx.x + gridDim.x) < items) issue(blockIdx.x + gridDim.x, true);
  unsigned phase = 0;
  constexpr int kEdW = (S::N + S::THREADS - 1) / S::THREADS;  // gx values of the row above, per thread
#pragma unroll 1
  for (int w = blockIdx.x; w < items; w += gridDim.x, phase ^= 1u) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    if (TRI && !ADJ && g == 0 && tid == 0)  // the sweep's count of finished blocks for this field starts at 0
      reinterpret_cast<unsigned*>(reinterpret_cast<double*>(partial) + (size_t)field * (kMaxRowBlocks / 2) + kTriCnt)[0] = 0u;
    float gxa[EDIT == kEditThreshold ? kEdW : 1];
    if constexpr (EDIT == kEditThreshold) {
      const int r0 = g * RW;
      const T* src = gx + field * fe + (size_t)(r0 > 0 ? r0 - 1 : 0) * A.W;
#pragma unroll
      for (int q = 0; q < kEdW; ++q) {
        const int j = tid + q * S::THREADS;
        gxa[q] = (r0 > 0 && j < A.W) ? f_to_f(src[j]) : 0.0f;
      }
    }
    const bool landed = mbar_wait(&bar, phase);
    if (__syncthreads_or(!landed)) {  // the copies never completed: report, let them drain, stop
      if (tid == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&bar, phase);
      return;
    }
    if constexpr (EDIT == kEditThreshold) {
      const float t2 = t2s[field];
      const int r0 = g * RW, nx = (A.H - r0) < RW ? (A.H - r0) : RW;
      const T zero = f_from_f<T>(0.0f);
      // staged pixels (r0 + i, j): gx in sgx row i, gy in sgy row i + 1; rows are
      // 16-byte multiples, so 16 bytes (VE pixels) at a time
      constexpr int VE = 16 / (int)sizeof(T);
      const int wv = A.W / VE;
      for (int idx = tid; idx < nx * wv; idx += S::THREADS) {
        const int i = idx / wv, jv = idx - i * wv;
        uint4* xp = reinterpret_cast<uint4*>(sgx + (size_t)i * A.W) + jv;
        uint4* yp = reinterpret_cast<uint4*>(sgy + (size_t)(i + 1) * A.W) + jv;
        uint4 xv = *xp, yv = *yp;
        T* xe = reinterpret_cast<T*>(&xv);
        T* ye = reinterpret_cast<T*>(&yv);
        bool any = false;
#pragma unroll
        for (int e2 = 0; e2 < VE; ++e2)
          if (edit_mag2(f_to_f(xe[e2]), f_to_f(ye[e2])) < t2) {
            xe[e2] = zero;
            ye[e2] = zero;
            any = true;
          }
        if (any) {
          *xp = xv;
          *yp = yv;
        }
      }
      if (r0 > 0) {  // gy of the row above (sgy row 0)
#pragma unroll
        for (int q = 0; q < kEdW; ++q) {
          const int j = tid + q * S::THREADS;
          if (j < A.W && edit_mag2(gxa[q], f_to_f(sgy[j])) < t2) sgy[j] = zero;
        }
      }
      __syncthreads();
    }
    float2 v[S::R1];
    if (ADJ && act) {
      // z = Crop^T(grad_out): rows ia, ib at torus rows p + ia, p + ib, columns
      // j < W at p + j; and the row pair's sum for the (sum grad_out) e_00 term,
      // compensated in FP32 (Knuth's TwoSum: the sum and the exact rounding
      // errors), so no FP64 work (scarce on this part) runs per value
      const int ia = g * RW + 2 * f, ib = ia + 1;
      const bool ha = ia < A.H, hb = ib < A.H;
      const T* xa = sgx + (size_t)(2 * f) * A.W;
      const T* xb = xa + A.W;
      float sum = 0.0f, err = 0.0f;
#pragma unroll
      for (int r = 0; r < S::R1; ++r) {
        const int j = t + S::R2 * r - kP;
        const bool sure = (S::R2 * r >= kP) && (S::R2 * r + S::R2 - 1 - kP < S::WMIN);
        const bool c1 = sure || (j >= 0 && j < A.W);
        const float a = (ha && c1) ? f_to_f(xa[j]) : 0.0f, b = (hb && c1) ? f_to_f(xb[j]) : 0.0f;
        v[r] = make_float2(a, b);
        sum = two_sum_acc(sum, a, err);
        sum = two_sum_acc(sum, b, err);
      }
      red[tid] = make_float2(sum, err);
    } else if (act) {
      const int r0 = g * RW, ia = r0 + 2 * f, ib = ia + 1;
      const bool ha = ia < A.H, hb = ib < A.H, hm = ia >= 1;  // rows present (ia - 1 < H always)
      const bool sa = ia < A.nrows, sb = ib < A.nrows;         // rows inside the support
      const T* xa = sgx + (size_t)(2 * f) * A.W;
      const T* xb = xa + A.W;
      const T* ym = sgy + (size_t)(2 * f) * A.W;  // gy row ia - 1
      const T* ya = ym + A.W;
      const T* yb = ya + A.W;
#pragma unroll
      for (int r = 0; r < S::R1; ++r) {
        const int j = t + S::R2 * r - kP;
        // columns j - 1 .. j inside [0, W) for every t and every width padding to N
        const bool sure = (S::R2 * r >= kP + 1) && (S::R2 * r + S::R2 - 1 - kP < S::WMIN);
        const bool c1 = sure || (j >= 0 && j < A.W), c0 = sure || (j >= 1 && j - 1 < A.W);
        const bool inj = sure || (j >= 0 && j < A.ncols);
        const float xa1 = (ha && c1) ? f_to_f(xa[j]) : 0.0f, xa0 = (ha && c0) ? f_to_f(xa[j - 1]) : 0.0f;
        const float xb1 = (hb && c1) ? f_to_f(xb[j]) : 0.0f, xb0 = (hb && c0) ? f_to_f(xb[j - 1]) : 0.0f;
        const float ya1 = (ha && c1) ? f_to_f(ya[j]) : 0.0f, yb1 = (hb && c1) ? f_to_f(yb[j]) : 0.0f;
        const float ym1 = (hm && c1) ? f_to_f(ym[j]) : 0.0f;
        const float la = (xa1 - xa0) + (ya1 - ym1);
        const float lb = (xb1 - xb0) + (yb1 - ya1);
        v[r] = make_float2((sa && inj) ? la : 0.0f, (sb && inj) ? lb : 0.0f);
      }
    }
    __syncthreads();  // every staged row read: the buffers become the exchange buffers
    if (ADJ && act && t == 0) {
      // the row pair's sum over its threads in order (compensated), stored in FP64
      float sp = 0.0f, ep = 0.0f;
      for (int k = 0; k < S::T; ++k) {
        const float2 e = red[f * S::T + k];
        sp = two_sum_acc(sp, e.x, ep);
        ep = __fadd_rn(ep, e.y);
      }
      reinterpret_cast<double*>(partial)[(size_t)field * (kMaxRowBlocks / 2) + g * S::F + f] = (double)sp + (double)ep;
    }
    if (act) {
      dft_reg<S::R1, -1>(v);
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();
    if (act && t < S::JSPAN) {
#pragma unroll
      for (int jj = 0; jj < S::J2; ++jj) {
        const int j = t + S::R2 * jj;
        float2 u[S::R2];
        u[0] = mybuf[j];
#pragma unroll
        for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[j + S::R1P * r], tw2[j * S::R2 + r]);
        dft_reg<S::R2, -1>(u);
#pragma unroll
        for (int s2 = 0; s2 < S::R2; ++s2) mybuf2[j + S::R1 * s2] = u[s2];
      }
    }
    __syncthreads();  // stage-2 results visible
    if constexpr (TRI) {
      tri_store_item<S, ADJ>(buf2, spec, tri, cc, field, g, A);
    } else {
    if (g == 0) {
      float2* Sz = spec + (size_t)field * A.Nh * A.ldM;
      const int nz = A.M - A.nrows;
      for (int idx = tid; idx < A.Nh * nz; idx += blockDim.x) {
        const int k = idx / nz, q = idx - k * nz;
        Sz[(size_t)k * A.ldM + (q < kP ? q : q + A.nrows)] = make_float2(0.0f, 0.0f);
      }
    }
    const int ra = g * 2 * S::F + 2 * uf;
    if (uact && ra < A.nrows) {
      float2* Sp = spec + (size_t)field * A.Nh * A.ldM + A.p + ra;
      const float2* zb = buf2 + uf * S::NO;
      const bool two = ra + 1 < A.nrows, vec = ((A.p + ra) & 1) == 0;
      for (int k = uk0; k < A.Nh; k += S::T) {
        const float2 zk = zb[k], zm = zb[k == 0 ? 0 : S::N - k];
        const float2 xa = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 xb = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        float2* dst = Sp + (size_t)k * A.ldM;
        if (two && vec) {
          *reinterpret_cast<float4*>(dst) = make_float4(xa.x, xa.y, xb.x, xb.y);
        } else {
          dst[0] = xa;
          if (two) dst[1] = xb;
        }
      }
    }
    }
    fence_proxy_async_smem();  // this thread's accesses of the buffers precede the next bulk copies
    __syncthreads();
    if (tid == 0 && w + (int)gridDim.x < items) issue(w + gridDim.x, false);
    if (tid == 0 && w + 2 * (int)gridDim.x < items) issue(w + 2 * gridDim.x, true);
  }
}

// ---------------------------------------------------------------------------
// pass B: column transform, Green multiply, inverse column transform, over
// items (field, block of C columns); persistent. Thread tid = t C + c works on
// column c of the block, so a warp's loads and stores cover whole 32-byte
// sectors of C neighbouring columns: the spectrum columns are read straight
// into registers (the next item's columns are prefetched into L2 meanwhile)
// and the result rows p .. p+H-1 (adjoint: p .. p+H) are written row-major
// straight from registers. The block's Green columns arrive by bulk copy,
// issued one item ahead.
// ---------------------------------------------------------------------------
// adjoint: sum(grad_out) of each field from its row-pair FP64 sums, lane-strided
// then a fixed shuffle tree (the same order on every call), into the field's
// slot kAdjTotal for the column pass; one warp per field
constexpr int kAdjTotal = kMaxRowBlocks / 2 - 1;
static __global__ void __launch_bounds__(32) k_adj_total(double* __restrict__ partial, int zpairs) {
  double* pp = partial + (size_t)blockIdx.x * (kMaxRowBlocks / 2);
  double a = 0.0;
  for (int i = threadIdx.x; i < zpairs; i += 32) a += pp[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (threadIdx.x == 0) pp[kAdjTotal] = a;
}

// ---------------------------------------------------------------------------
// Recursive column solve, between the row passes: the carry sweep. A block
// takes 32 columns (one per lane) of one field; its kTriSeg warps cut the G
// bands into segments. With T_g = a^(rows of band g):
//   causal:     the carry into band g is c_g, c_{g+1} = e_g + T_g c_g around the
//               cycle, where the rows after the last band (tail) and above band 0
//               (pad) are zero: a^tail (c_G - prod T c_0) = (1 - a^M) y[M-1] -
//               ..., i.e. with P the sweep of the e_g from a zero carry,
//               y[M-1] = a^tail P_G / (1 - a^M) and c_0 = a^p y[M-1];
//   anticausal: the carry from below band g is q_g, q_{g-1} = e'_g + T_g q_g,
//               q_{G-1} = a^tail y'[0], y'[0] = a^p Q_{-1} / (1 - a^M) with Q the
//               sweep from a zero carry.
// Each warp sweeps its segment from zero carries (both directions); warps 0
// and 1 then sweep the segment totals (segment transfers a^(2F n) from the
// plan's FP64 power table) and close the cycle; every warp re-sweeps its
// segment from its true carries and writes c_g, q_g (the band sums are read
// twice, the second time from cache). Row 0 of the solved spectrum (a padding
// row, X = 0) is U[0][l] = C_l (a y[M-1] + y'[0]): the block's FP64 sum of
// w_l Re U[0][l] (w = 1 at l = N/2, else 2) is its partial of u[0,0], added in
// block order by the inverse row pass. Column 0 (b = 2, singular) is the 1D
// periodic Poisson problem with its mean removed (the reading G[0,0] = 0): the
// extra warp of block 0 solves it exactly in FP64 and writes it into S.
// ---------------------------------------------------------------------------
constexpr int kTriMaxM = 2112;  // column 0 of the longest supported column
constexpr int kTriSeg = kTriSegments;  // band segments (warps) per sweep block
constexpr int kTriTileMaxG = 160;      // bands whose sums a sweep block stages (80 KB)

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_exclusive_scan_d(double v) {
  const int lane = threadIdx.x & 31;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

// Column 0 of one field (warp-wide, FP64): d[r] = u[r+1] - u[r] has
// d[r] - d[r-1] = f[r] - mean(f); periodicity fixes d[-1] = -sum_r G[r] / M with
// G the prefix sums; u[0] = 0 (any constant is removed with u[0,0]: column 0
// adds w_0 U[0][0] = u[0] / N = 0 to it). fcol[p + i] holds column 0 of S row
// i (bulk copy of pass A's compact copy); each lane walks a contiguous run of
// torus rows; the solution (1/N folded in) replaces column 0 of S.
static __device__ __noinline__ void tri_column0(float2* __restrict__ spec, float* fcol, int field,
                                                const FastArgs& A, float x0) {
  const int lane = threadIdx.x & 31;
  float2* col = spec + (size_t)field * A.srows * A.ldY;
  const int nr = min(A.srows, A.M - A.p);  // S rows on the torus
  for (int r = lane; r < A.M; r += 32)
    if (r < A.p || r >= A.p + nr) fcol[r] = 0.0f;
  if (lane == 0) fcol[0] = x0;  // torus row 0 (the adjoint's -(sum grad_out) e_00; else 0)
  __syncwarp();
  const int run = (A.M + 31) / 32;
  const int r0 = min(lane * run, A.M), r1 = min(r0 + run, A.M);
  double s0 = 0.0;
  for (int r = r0; r < r1; ++r) s0 += (double)fcol[r];
  const double mean = warp_sum_d(s0) * A.invM;
  const double off = warp_exclusive_scan_d(s0 - mean * (double)(r1 - r0));
  double Gr = off, Gs = 0.0;
  for (int r = r0; r < r1; ++r) {
    Gr += (double)fcol[r] - mean;
    Gs += Gr;
  }
  const double D = -warp_sum_d(Gs) * A.invM;
  double u = warp_exclusive_scan_d(D * (double)(r1 - r0) + Gs);
  const double invN = A.invN;
  Gr = off;
  for (int r = r0; r < r1; ++r) {
    const int i = r - A.p;
    if (i >= 0 && i < nr) col[(size_t)i * A.ldY] = make_float2((float)(u * invN), 0.0f);
    Gr += (double)fcol[r] - mean;
    u += D + Gr;
  }
}

static __global__ void __launch_bounds__(32 * (kTriSeg + 1)) k_tri_carries(float2* __restrict__ spec,
                                                                          float2* __restrict__ tri,
                                                                          const float* __restrict__ cc,
                                                                          const float* __restrict__ powc,
                                                                          double* __restrict__ partial, FastArgs A) {
  __shared__ float2 seg_e[kTriSeg][kTriCols], seg_q[kTriSeg][kTriCols];  // segment totals, then carries
  __shared__ float2 y0s[kTriCols];
  __shared__ float yls[2 * kTriCols];
  __shared__ __align__(16) float fcol[kTriMaxM + 4];  // block 0: column 0 of S (compact copy)
  __shared__ __align__(8) uint64_t bar, tbar;
  extern __shared__ __align__(16) float2 tile[];  // the block's band sums when they fit (staged)
  const int kb = blockIdx.x, field = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = kb * kTriCols + lane;
  const bool col_ok = k >= 1 && k < A.Nh;
  // the adjoint's z has -(sum grad_out) at torus (0, 0): -s in every column of row 0
  const float sadj = A.adj ? (float)partial[(size_t)field * (kMaxRowBlocks / 2) + kAdjTotal] : 0.0f;
  const float2* gsums = tri_sums(tri, field, A) + (size_t)kb * 2 * A.G * kTriCols;  // [g][2][32], contiguous
  const bool staged = A.G <= kTriTileMaxG;
  const float2* sums = (staged ? tile : gsums) + lane;
  float2* carry = tri + (size_t)field * A.tri_field + k;  // [g][2][ldY]
  // column 0's compact copy for block 0's extra warp, in flight during the sweeps
  const int nr = min(A.srows, A.M - A.p);
  const unsigned cbytes = (unsigned)((nr * sizeof(float) + 15) & ~(size_t)15);
  if (kb == 0 && tid == 32 * kTriSeg) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, cbytes);
    bulk_copy(fcol + A.p, tri_col0(tri, field, A), cbytes, &bar);
  }
  if (staged) {  // the whole tile of band sums by one bulk copy
    if (tid == 0) {
      mbar_init(&tbar, 1);
      bulk_load(tile, gsums, (unsigned)(2 * A.G * kTriCols * sizeof(float2)), &tbar);
    }
    __syncthreads();
    const bool landed = mbar_wait(&tbar, 0);
    if (__syncthreads_or(!landed)) {  // the copy never completed: report, let it drain, stop
      if (tid == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&tbar, 0);
      if (kb == 0 && tid == 32 * kTriSeg) mbar_wait(&bar, 0);
      return;
    }
  }
  float4 c03 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), c47 = c03;
  if (col_ok) {
    c03 = __ldg(reinterpret_cast<const float4*>(cc + (size_t)k * 8));
    c47 = __ldg(reinterpret_cast<const float4*>(cc + (size_t)k * 8) + 1);
  }
  const float a = c03.y, C = c03.z, Tb = c03.w, Tl = c47.x, Tp = c47.y, inv = c47.z, Tt = c47.w;
  const int per = (A.G + kTriSeg - 1) / kTriSeg;
  const int g0 = min(warp * per, A.G), g1 = min(g0 + per, A.G);
  // phase 1: each segment from zero carries
  if (warp < kTriSeg) {
    float2 t = make_float2(0.0f, 0.0f), q = t;
    if (col_ok) {
#pragma unroll 4
      for (int g = g0; g < g1; ++g) {
        const float T = (g == A.G - 1) ? Tl : Tb;
        const float2 e = sums[(size_t)g * 2 * kTriCols];
        t = __ffma2_rn(make_float2(T, T), t, e);
      }
#pragma unroll 4
      for (int g = g1 - 1; g >= g0; --g) {
        const float T = (g == A.G - 1) ? Tl : Tb;
        const float2 e = sums[(size_t)g * 2 * kTriCols + kTriCols];
        q = __ffma2_rn(make_float2(T, T), q, e);
      }
    }
    seg_e[warp][lane] = t;
    seg_q[warp][lane] = q;
  }
  __syncthreads();
  // phase 2: the segment totals around the cycle (warp 0 causal, warp 1 anticausal)
  if (warp < 2 && col_ok) {
    float Ts[kTriSeg];  // transfer of segment s: a^(rows of its bands), all loaded at once
#pragma unroll
    for (int s2 = 0; s2 < kTriSeg; ++s2) {
      const int b0 = min(s2 * per, A.G), b1 = min(b0 + per, A.G);
      Ts[s2] = (b1 <= b0) ? 1.0f
                          : (b1 < A.G ? __ldg(powc + (size_t)(b1 - b0) * A.ldY + k)
                                      : __ldg(powc + (size_t)(b1 - b0 - 1) * A.ldY + k) * Tl);
    }
    auto seg_T = [&](int s2) { return Ts[s2]; };
    if (warp == 0) {
      float2 t = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int s = 0; s < kTriSeg; ++s) {
        const float T = seg_T(s);
        const float2 e = seg_e[s][lane];
        t = make_float2(fmaf(T, t.x, e.x), fmaf(T, t.y, e.y));
      }
      const float2 yl = make_float2(Tt * t.x * inv, Tt * t.y * inv);  // y[M-1]
      float2 c = make_float2(Tp * yl.x, Tp * yl.y);                   // y[p-1]: carry into band 0
      if (A.adj) c.x -= (Tp / a) * sadj * inv;  // row 0's -s, carried a^(p-1) down
#pragma unroll
      for (int s = 0; s < kTriSeg; ++s) {
        const float T = seg_T(s);
        const float2 e = seg_e[s][lane];
        seg_e[s][lane] = c;
        c = make_float2(fmaf(T, c.x, e.x), fmaf(T, c.y, e.y));
      }
      yls[lane] = yl.x;
    } else {
      float2 q = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int s = kTriSeg - 1; s >= 0; --s) {
        const float T = seg_T(s);
        const float2 e = seg_q[s][lane];
        q = make_float2(fmaf(T, q.x, e.x), fmaf(T, q.y, e.y));
      }
      float2 y0 = make_float2(Tp * q.x * inv, Tp * q.y * inv);  // y'[0]
      if (A.adj) y0.x = (Tp * q.x - sadj) * inv;
      float2 c = make_float2(Tt * y0.x, Tt * y0.y);                   // carry from below the last band
#pragma unroll
      for (int s = kTriSeg - 1; s >= 0; --s) {
        const float T = seg_T(s);
        const float2 e = seg_q[s][lane];
        seg_q[s][lane] = c;
        c = make_float2(fmaf(T, c.x, e.x), fmaf(T, c.y, e.y));
      }
      y0s[lane] = y0;
    }
  }
  __syncthreads();
  // phase 3: each segment again from its true carries; the carries go out
  if (warp < kTriSeg && col_ok) {
    float2 c = seg_e[warp][lane];
#pragma unroll 4
    for (int g = g0; g < g1; ++g) {
      const float T = (g == A.G - 1) ? Tl : Tb;
      const float2 e = sums[(size_t)g * 2 * kTriCols];
      carry[(size_t)(2 * g) * A.ldY] = c;
      c = __ffma2_rn(make_float2(T, T), c, e);
    }
    float2 q = seg_q[warp][lane];
#pragma unroll 4
    for (int g = g1 - 1; g >= g0; --g) {
      const float T = (g == A.G - 1) ? Tl : Tb;
      const float2 e = sums[(size_t)g * 2 * kTriCols + kTriCols];
      carry[(size_t)(2 * g + 1) * A.ldY] = q;
      q = __ffma2_rn(make_float2(T, T), q, e);
    }
  }
  if (warp == 0 && !A.adj) {  // u[0,0] (the adjoint has no offset)
    double acc = 0.0;
    if (col_ok) acc = (2 * k == A.N ? 1.0 : 2.0) * (double)(C * fmaf(a, yls[lane], y0s[lane].x));
    acc = warp_sum_d(acc);
    double* pp = partial + (size_t)field * (kMaxRowBlocks / 2);
    unsigned done = 0;
    if (lane == 0) {
      pp[kb] = acc;
      __threadfence();  // this partial is visible before the count says so
      done = atomicAdd(reinterpret_cast<unsigned*>(pp + kTriCnt), 1u);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done == (unsigned)gridDim.x - 1) {
      // the field's last sweep block: u[0,0] from every block's partial,
      // lane-strided then a fixed shuffle tree (the same order on every call)
      __threadfence();
      double s2 = 0.0;
      for (int i = lane; i < (int)gridDim.x; i += 32) s2 += __ldcg(pp + i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o);
      if (lane == 0) pp[kTriU00] = s2;
    }
  }
  if (warp == kTriSeg && kb == 0) {
    const bool landed = mbar_wait(&bar, 0);
    if (!landed) {  // the copy never completed: report, let it drain, stop
      if (lane == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&bar, 0);
      return;
    }
    tri_column0(spec, fcol, field, A, -sadj);
  }
}

// The carry sweep for fields of at most kTriRegG bands: one warp per (field,
// block of 32 columns), one column per lane, all of the block's band sums in
// registers (one round of loads per direction), each direction swept from a
// zero carry and then from the true carries, as above; no shared-memory
// staging and no block barriers. The warp of column block 0 then solves
// column 0 exactly (fcol: M + 4 floats of shared memory per warp), and each
// field's last warp to finish combines the u[0,0] partials.
constexpr int kTriRegG = 32;
constexpr int kTriRegWarps = 8;
static __global__ void __launch_bounds__(32 * kTriRegWarps, 2) k_tri_carries_reg(float2* __restrict__ spec,
                                                                           float2* __restrict__ tri,
                                                                           const float* __restrict__ cc,
                                                                           double* __restrict__ partial, FastArgs A,
                                                                           int nkb) {
  extern __shared__ __align__(16) float fcols[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int task = blockIdx.x * kTriRegWarps + warp;
  if (task >= A.nf * nkb) return;
  const int field = task / nkb, kb = task - field * nkb;
  const int k = kb * kTriCols + lane;
  const bool col_ok = k >= 1 && k < A.Nh;
  const int G = A.G;
  // the adjoint's z has -(sum grad_out) at torus (0, 0): -s in every column of row 0
  const float sadj = A.adj ? (float)partial[(size_t)field * (kMaxRowBlocks / 2) + kAdjTotal] : 0.0f;
  const float2* sums = tri_sums(tri, field, A) + (size_t)kb * 2 * G * kTriCols + lane;  // [g][2][32]
  float2* carry = tri + (size_t)field * A.tri_field + k;                                 // [g][2][ldY]
  double acc = 0.0;
  if (col_ok) {
    const float4 c03 = __ldg(reinterpret_cast<const float4*>(cc + (size_t)k * 8));
    const float4 c47 = __ldg(reinterpret_cast<const float4*>(cc + (size_t)k * 8) + 1);
    const float a = c03.y, C = c03.z, Tb = c03.w, Tl = c47.x, Tp = c47.y, inv = c47.z, Tt = c47.w;
    float2 yl, y0;
    {  // causal: the band sums in registers, from a zero carry, close the cycle, carries out
      float2 e[kTriRegG];
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) e[g] = sums[(size_t)g * 2 * kTriCols];
      float2 t = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          t = __ffma2_rn(make_float2(T, T), t, e[g]);
        }
      yl = make_float2(Tt * t.x * inv, Tt * t.y * inv);  // y[M-1]
      float2 c = make_float2(Tp * yl.x, Tp * yl.y);     // carry into band 0
      if (A.adj) c.x -= (Tp / a) * sadj * inv;          // row 0's -s, carried a^(p-1) down
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          carry[(size_t)(2 * g) * A.ldY] = c;
          c = __ffma2_rn(make_float2(T, T), c, e[g]);
        }
    }
    {  // anticausal, the same way up the bands
      float2 ep[kTriRegG];
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) ep[g] = sums[(size_t)g * 2 * kTriCols + kTriCols];
      float2 q = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int g = kTriRegG - 1; g >= 0; --g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          q = __ffma2_rn(make_float2(T, T), q, ep[g]);
        }
      y0 = make_float2(Tp * q.x * inv, Tp * q.y * inv);  // y'[0]
      if (A.adj) y0.x = (Tp * q.x - sadj) * inv;
      float2 c = make_float2(Tt * y0.x, Tt * y0.y);     // carry from below the last band
#pragma unroll
      for (int g = kTriRegG - 1; g >= 0; --g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          carry[(size_t)(2 * g + 1) * A.ldY] = c;
          c = __ffma2_rn(make_float2(T, T), c, ep[g]);
        }
    }
    acc = (2 * k == A.N ? 1.0 : 2.0) * (double)(C * fmaf(a, yl.x, y0.x));
  }
  acc = warp_sum_d(acc);
  double* pp = partial + (size_t)field * (kMaxRowBlocks / 2);
  if (kb == 0) {  // column 0, from the compact copy of S's column 0
    float* fcol = fcols + (size_t)warp * (A.M + 4);
    const int nr = min(A.srows, A.M - A.p);
    const float* c0 = tri_col0(tri, field, A);
    for (int i = lane; i < nr; i += 32) fcol[A.p + i] = c0[i];
    __syncwarp();
    tri_column0(spec, fcol, field, A, -sadj);
  }
  if (A.adj) return;  // u[0,0]: the adjoint has no offset
  unsigned done = 0;
  if (lane == 0) {
    pp[kb] = acc;
    __threadfence();  // this partial is visible before the count says so
    done = atomicAdd(reinterpret_cast<unsigned*>(pp + kTriCnt), 1u);
  }
  done = __shfl_sync(0xffffffffu, done, 0);
  if (done == (unsigned)nkb - 1) {
    // the field's last warp: u[0,0] from every column block's partial,
    // lane-strided then a fixed shuffle tree (the same order on every call)
    __threadfence();
    double s2 = 0.0;
    for (int i = lane; i < nkb; i += 32) s2 += __ldcg(pp + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o);
    if (lane == 0) pp[kTriU00] = s2;
  }
}

template <class S, int MODE>
__global__ void __launch_bounds__(S::THREADS, S::MINB) k_fast_cols(const float2* __restrict__ spec, float2* __restrict__ Y,
                                                          const float* __restrict__ GT, const float2* __restrict__ twg,
                                                          float* __restrict__ partial, FastArgs A) {
  extern __shared__ __align__(16) float2 sm[];
  float* gsm = reinterpret_cast<float*>(sm);                       // [C][GS] Green columns of the item
  float2* twF = reinterpret_cast<float2*>(gsm + S::C * S::GS);     // [R1][TWF_STRIDE]: w_M^(r j), j < R1, r < R2
  float2* twI = twF + S::R1 * S::TWF_STRIDE;                       // [R2][TWI_STRIDE]: w_M^(r j), j < R2, r < R1
  float2* xbuf = twI + S::R2 * S::TWI_STRIDE;                      // [C][MP] exchange
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int c = tid % S::C, t = tid / S::C;
  const bool act = t < S::R2, act2 = t < S::R1;
  const int items = A.nf * A.nparts;
  const int yrows = (MODE == 2) ? A.H + 1 : A.H;
  float2* mybuf = xbuf + c * S::MP;
  const float* gcol = gsm + c * S::GS;
  auto ncols_of = [&](int blk) { return (A.Nh - blk * S::C) < S::C ? (A.Nh - blk * S::C) : S::C; };
  auto issue_green = [&](int w) {  // one thread
    const int blk = w % A.nparts;
    const unsigned gb = (unsigned)(ncols_of(blk) * A.ldM * sizeof(float));
    bulk_load(gsm, GT + (size_t)blk * S::C * A.ldM, gb, &bar);
  };
  auto prefetch_spec = [&](int w) {  // one thread: the item's spectrum columns into L2
    const int field = w / A.nparts, blk = w - field * A.nparts;
    l2_prefetch(spec + ((size_t)field * A.Nh + (size_t)blk * S::C) * A.ldM,
                (unsigned)(ncols_of(blk) * A.ldM * sizeof(float2)));
  };
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    twF[j * S::TWF_STRIDE + r] = twg[r * j];
  }
  for (int i = tid; i < S::R2 * S::R1; i += blockDim.x) {
    const int j = i / S::R1, r = i - j * S::R1;
    twI[j * S::TWI_STRIDE + r] = twg[r * j];
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    if ((int)blockIdx.x < items) issue_green(blockIdx.x);
  }
  __syncthreads();  // barrier initialised, twiddles in place
  unsigned phase = 0;
#pragma unroll 1
  for (int w = blockIdx.x; w < items; w += gridDim.x, phase ^= 1u) {
    const int field = w / A.nparts, blk = w - field * A.nparts;
    const int l = blk * S::C + c;
    const bool colok = l < A.Nh;
    if (tid == 0 && w + (int)gridDim.x < items) prefetch_spec(w + gridDim.x);
    // rows outside the support were zeroed by the row pass
    float2 v[S::R1];
    {
      const float2* col = spec + ((size_t)field * A.Nh + (colok ? l : 0)) * A.ldM;
#pragma unroll
      for (int r = 0; r < S::R1; ++r) v[r] = (act && colok) ? col[t + S::R2 * r] : make_float2(0.0f, 0.0f);
    }
    if (MODE == 2) {
      // adjoint: z = Crop^T(grad_out) - (sum grad_out) e_00; the row DFT of the
      // second term is -sum in every column, at torus row 0 (the sum from
      // k_adj_total); the threads with t = 0 are lanes 0 .. C-1 of warp 0.
      if (t == 0) {
        const double a = reinterpret_cast<const double*>(partial)[(size_t)field * (kMaxRowBlocks / 2) + kAdjTotal];
        v[0] = make_float2((float)(-a), 0.0f);
      }
    }
    if (act) dft_reg<S::R1, -1>(v);
    __syncthreads();  // the previous item's reads of the exchange are done
    if (act) {
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1 + s2] = v[s2];
    }
    __syncthreads();
    float2 u[S::R2];
    if (act2) {
      u[0] = mybuf[t];
#pragma unroll
      for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[t + S::R1 * r], twF[t * S::TWF_STRIDE + r]);
      dft_reg<S::R2, -1>(u);
    }
    const bool landed = mbar_wait(&bar, phase);
    if (act2) {
      // bins k = t + R1 s: multiply by the real Green spectrum (Eq. 23)
#pragma unroll
      for (int s2 = 0; s2 < S::R2; ++s2) u[s2] = cscale(u[s2], gcol[t + S::R1 * s2]);
      // inverse stage 1 (span 1): butterfly t takes exactly the bins t + R1 r held here
      dft_reg<S::R2, +1>(u);
    }
    fence_proxy_async_smem();  // this thread's reads of the Green columns precede the next bulk copy
    if (__syncthreads_or(!landed)) {  // the copy never completed: report, let it drain, stop
      if (tid == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&bar, phase);
      return;
    }
    if (tid == 0 && w + (int)gridDim.x < items) issue_green(w + gridDim.x);
    if (act2) {
#pragma unroll
      for (int s2 = 0; s2 < S::R2; ++s2) mybuf[t * (S::R2 + 1) + s2] = u[s2];  // pad(t R2 + s2), s2 < R2
    }
    __syncthreads();
    if (act) {
      // pad(t + R2 r) = t + (R2 + 1) r for t < R2
      v[0] = mybuf[t];
#pragma unroll
      for (int r = 1; r < S::R1; ++r) v[r] = cmul(mybuf[t + (S::R2 + 1) * r], cconj(twI[t * S::TWI_STRIDE + r]));
      dft_reg<S::R1, +1>(v);
    }
    if (MODE != 2 && tid < 32) {
      // u[0,0] = sum over the row-0 spectrum, weight 1 at l = 0 and N/2, 2
      // elsewhere; FP64, columns added in order (an error in u[0,0] shifts
      // every output pixel)
      const double cv = (tid < S::C && colok) ? ((l == 0 || 2 * l == A.N) ? (double)v[0].x : 2.0 * (double)v[0].x)
                                              : 0.0;
      double s2 = 0.0;
#pragma unroll
      for (int cc = 0; cc < S::C; ++cc) s2 += __shfl_sync(0xffffffffu, cv, cc);
      if (tid == 0) reinterpret_cast<double*>(partial)[(size_t)field * (kMaxRowBlocks / 2) + blk] = s2;
    }
    if (act && colok) {
      float2* Yc = Y + (size_t)field * yrows * A.ldY + l;
#pragma unroll
      for (int r = 0; r < S::R1; ++r) {
        const int i = t + S::R2 * r - A.p;  // image row of torus row t + R2 r
        if (i >= 0 && i < yrows) Yc[(size_t)i * A.ldY] = v[r];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// pass C: inverse row transforms of the row-major spectrum Y with the
// Hermitian extension formed on load, offset, crop and cast. Persistent over
// (field, group of F output row pairs). The 2F rows of Y an item needs are one
// contiguous bulk copy into the exchange buffer, completed on an mbarrier; the
// copy for the next item is issued as soon as this item's stage-2 inputs are
// in registers, so it overlaps the stage-2 transforms and the output stores.
// ---------------------------------------------------------------------------
// Recursive column solve, pass C side: the 2F staged rows of band g (row-major
// spectrum S) become rows of the solved spectrum U in place. Per column l >= 1,
// from the band's two staged carries: the causal recursion down the band and
// the anticausal one up it, U = C_l (y + y' - X). Column 0 already holds its
// exact solution. Rows past the torus (band rows >= nb) are left alone: they
// are below every image row.
template <class S>
__device__ __forceinline__ void tri_solve_band(float2* buf, const float2* cbuf, const float* __restrict__ cc, int g,
                                               const FastArgs& A) {
  constexpr int RW = 2 * S::F;
  const int nb = min(RW, A.M - A.p - g * RW);
  if constexpr (S::SHORT) {
    // short rows: one column per thread (the band's RW values of a column pair
    // would not fit the registers of four blocks per SM)
    const float2* dcs = reinterpret_cast<const float2*>(cc + (size_t)A.Nh * 8);  // (delta, C) per column
    for (int k = 1 + threadIdx.x; k < A.Nh; k += blockDim.x) {
      const float2 dc = __ldg(dcs + k);
      float2 yc = cbuf[k], ya = cbuf[S::LDY + k];
      float2* col = buf + k;
      float2 x[RW];
#pragma unroll
      for (int r = 0; r < RW; ++r) x[r] = col[(size_t)r * S::LDY];
#pragma unroll
      for (int r = 0; r < RW; ++r)
        if (r < nb) {
          yc = tri_step(x[r], yc, dc.x);
          col[(size_t)r * S::LDY] = yc;
        }
#pragma unroll
      for (int r = RW - 1; r >= 0; --r)
        if (r < nb) {
          ya = tri_step(x[r], ya, dc.x);
          col[(size_t)r * S::LDY] = cscale(csub(cadd(col[(size_t)r * S::LDY], ya), x[r]), dc.y);
        }
    }
  } else {
  // thread t takes the column pair (2j, 2j + 1), 16-byte shared-memory accesses;
  // column 0 (already solved) and columns >= Nh pass through unchanged
  for (int j = threadIdx.x; 2 * j < A.Nh; j += blockDim.x) {
    const int k0 = 2 * j;
    const bool v0 = k0 >= 1, v1 = k0 + 1 < A.Nh;
    // (delta, C) of both columns in one coalesced 16-byte load (the plan's compact table)
    const float4 dc = __ldg(reinterpret_cast<const float4*>(cc + (size_t)A.Nh * 8) + j);
    const float dl0 = dc.x, C0 = v0 ? dc.y : 1.0f, dl1 = dc.z, C1 = v1 ? dc.w : 1.0f;
    const float4 yc4 = reinterpret_cast<const float4*>(cbuf)[j];
    const float4 ya4 = reinterpret_cast<const float4*>(cbuf + S::LDY)[j];
    float2 yc0 = make_float2(yc4.x, yc4.y), yc1 = make_float2(yc4.z, yc4.w);
    float2 ya0 = make_float2(ya4.x, ya4.y), ya1 = make_float2(ya4.z, ya4.w);
    float4* col = reinterpret_cast<float4*>(buf) + j;
    float4 x[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) x[r] = col[(size_t)r * (S::LDY / 2)];
#pragma unroll
    for (int r = 0; r < RW; ++r)
      if (r < nb) {
        yc0 = tri_step(make_float2(x[r].x, x[r].y), yc0, dl0);
        yc1 = tri_step(make_float2(x[r].z, x[r].w), yc1, dl1);
        col[(size_t)r * (S::LDY / 2)] = make_float4(yc0.x, yc0.y, yc1.x, yc1.y);
      }
#pragma unroll
    for (int r = RW - 1; r >= 0; --r)
      if (r < nb) {
        ya0 = tri_step(make_float2(x[r].x, x[r].y), ya0, dl0);
        ya1 = tri_step(make_float2(x[r].z, x[r].w), ya1, dl1);
        const float4 y = col[(size_t)r * (S::LDY / 2)];
        const float2 u0 = cscale(csub(cadd(make_float2(y.x, y.y), ya0), make_float2(x[r].x, x[r].y)), C0);
        const float2 u1 = cscale(csub(cadd(make_float2(y.z, y.w), ya1), make_float2(x[r].z, x[r].w)), C1);
        float4 u = make_float4(u0.x, u0.y, u1.x, u1.y);
        if (!v0) {  // column 0 keeps its exact solution
          u.x = x[r].x;
          u.y = x[r].y;
        }
        col[(size_t)r * (S::LDY / 2)] = u;
      }
  }
  }
}

// Per-field statistics of the stored output (colour correction, Eq. 25): item
// g of a field writes (sum x, sum x^2) of its stored values in FP64 at
// partial (as doubles) + field * kMaxRowBlocks / 2 + kStatsOff + 2 g.
constexpr int kStatsOff = 160;

template <class S, typename T, bool TRI, bool STATS>
__global__ void __launch_bounds__(S::THREADS, S::MINB_INV) k_fast_rows_inv(const float2* __restrict__ Y,
                                                              float* __restrict__ partial, T* __restrict__ out,
                                                              const float2* __restrict__ twg, FastArgs A,
                                                              const float2* __restrict__ tri,
                                                              const float* __restrict__ cc) {
  extern __shared__ __align__(16) float2 sm[];
  float2* tw2 = sm;
  float2* buf = sm + S::R1 * S::R2;  // staged rows of Y (TRI: of S) [2F][ldY], then the stage-1 exchange
  float2* cbuf = sm + S::CBUF;        // TRI: the band's two carries [2][LDY]
  __shared__ float u00s[2];
  __shared__ __align__(8) uint64_t bar;
  constexpr int RW = 2 * S::F;       // rows of Y per item
  const int tid = threadIdx.x;
  const int f = tid / S::T, t = tid - f * S::T;
  const bool act = f < S::F;
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    tw2[i] = twg[r * j];
  }
  float2* mybuf = buf + (act ? f : 0) * S::NP;
  const int half = S::N / 2;
  const int items = A.nf * A.ngroups;
  // one thread: stage the rows of item w (prefetch: only start fetching them
  // into L2, for the copy one item later)
  auto issue = [&](int w, bool prefetch) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    const int r0 = g * RW, nr = (A.H - r0) < RW ? (A.H - r0) : RW;
    if constexpr (TRI) {  // the whole band of S (its rows past the image feed the recursions) and its carries
      const unsigned rb = (unsigned)(RW * A.ldY * sizeof(float2)), cb = (unsigned)(2 * A.ldY * sizeof(float2));
      const float2* ss = Y + ((size_t)field * A.srows + r0) * A.ldY;
      const float2* cs = tri + (size_t)field * A.tri_field + (size_t)g * 2 * A.ldY;
      if (prefetch) {
        l2_prefetch(ss, rb);
        l2_prefetch(cs, cb);
        return;
      }
      mbar_expect_tx(&bar, rb + cb);
      if (A.l2res)  // the band's last read
        bulk_copy_hint(buf, ss, rb, &bar, l2_policy_evict_first());
      else
        bulk_copy(buf, ss, rb, &bar);
      bulk_copy(cbuf, cs, cb, &bar);
    } else {
      const float2* ys = Y + ((size_t)field * A.H + r0) * A.ldY;
      const unsigned nb = (unsigned)(nr * A.ldY * sizeof(float2));
      if (prefetch)
        l2_prefetch(ys, nb);
      else
        bulk_load(buf, ys, nb, &bar);
    }
  };
  // warp 0 loads the u[0,0] partial sums of the next item while this one is
  // transformed (lane-strided, the same order as a plain loop over them); with
  // the recursive column solve the carry sweep has already combined them into
  // the field's u[0,0] (kTriU00), one value to load
  constexpr int KPF = TRI ? 1 : 5;
  double pf[KPF];
  auto prefetch = [&](int w) {
    if (tid < 32 && w < items) {
      const double* pp = reinterpret_cast<const double*>(partial) + (size_t)(w / A.ngroups) * (kMaxRowBlocks / 2);
      if constexpr (TRI) {
        pf[0] = tid == 0 ? pp[kTriU00] : 0.0;
      } else {
#pragma unroll
        for (int k = 0; k < KPF; ++k) pf[k] = (tid + 32 * k < A.nparts) ? pp[tid + 32 * k] : 0.0;
      }
    }
  };
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < items) issue(blockIdx.x, false);
  if (tid == 0 && (int)(blockIdx.x + gridDim.x) < items) issue(blockIdx.x + gridDim.x, true);
  prefetch(blockIdx.x);
  int parity = 0;
  unsigned phase = 0;
#pragma unroll 1
  for (int w = blockIdx.x; w < items; w += gridDim.x, parity ^= 1, phase ^= 1u) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    if constexpr (TRI) {
      if (tid == 0) u00s[parity] = (float)pf[0];
    } else if (tid < 32) {
      // u[0,0] from the column blocks' FP64 partial sums: lane-strided, then a
      // fixed shuffle tree (the same order on every call)
      double s2 = 0.0;
      if (A.nparts <= 32 * KPF) {
#pragma unroll
        for (int k = 0; k < KPF; ++k) s2 += pf[k];
      } else {
        const double* pp = reinterpret_cast<const double*>(partial) + (size_t)field * (kMaxRowBlocks / 2);
        for (int i = tid; i < A.nparts; i += 32) s2 += pp[i];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o);
      if (tid == 0) u00s[parity] = (float)s2;
    }
    const bool landed = mbar_wait(&bar, phase);
    if (__syncthreads_or(!landed)) {  // the copy never completed: report, let it drain, stop
      if (tid == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&bar, phase);
      if (tid == 0) bulk_store_wait();
      return;
    }
    if constexpr (TRI) {
      if (A.l2res)  // the band's rows of S are in shared memory and dead in global memory: drop their L2 lines
        l2_discard_range(Y + ((size_t)field * A.srows + (size_t)g * RW) * A.ldY, (size_t)RW * A.ldY * sizeof(float2),
                         tid, blockDim.x);
      tri_solve_band<S>(buf, cbuf, cc, g, A);
      __syncthreads();
    }
    const int ia = g * 2 * S::F + 2 * f, ib = ia + 1;
    const bool va = act && ia < A.H, vb = act && ib < A.H;
    const float2* ya_row = buf + (size_t)(va ? 2 * f : 0) * A.ldY;
    const float2* yb_row = buf + (size_t)(vb ? 2 * f + 1 : 0) * A.ldY;
    float2 v[S::R1];
#pragma unroll
    for (int r = 0; r < S::R1; ++r) {
      // l = t + R2 r with t < R2: whether l lies below or above N/2 is known at
      // compile time except for the one r whose range contains N/2
      const int l = t + S::R2 * r;
      const bool all_lo = S::R2 * r + S::R2 - 1 < half;
      const bool all_hi = S::R2 * r > half;
      const bool lo = all_lo || (!all_hi && l < half);
      const int src = lo ? l : S::N - l;
      float2 ya = va ? ya_row[src] : make_float2(0.0f, 0.0f);
      float2 yb = vb ? yb_row[src] : make_float2(0.0f, 0.0f);
      // bins 0 and N/2 are real in a real transform: drop their imaginary parts
      const bool may_edge = (r == 0) || (!all_lo && !all_hi);
      if (may_edge && (src == 0 || src == half)) {
        ya.y = 0.0f;
        yb.y = 0.0f;
      }
      v[r] = lo ? make_float2(ya.x - yb.y, ya.y + yb.x) : make_float2(ya.x + yb.y, yb.x - ya.y);
    }
    if (act) dft_reg<S::R1, +1>(v);
    __syncthreads();  // every staged row read: buf becomes the exchange buffer
    if (act) {
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();
    const bool act2 = act && t < S::JSPAN;
    const float u00 = u00s[parity];
    T* o = out + (size_t)field * A.H * A.W;
    // one stage-2 butterfly per thread: once its inputs are in registers the
    // exchange buffer is free, and the item's output rows are staged there
    // ([2F][W], the output's own row pitch) and leave by one bulk copy
    const bool stage = S::J2 == 1 && A.stage_out;
    T* srows = reinterpret_cast<T*>(buf);
    // STATS: this thread's stored values as float sums about its first value
    float st_sh = 0.0f, st_s = 0.0f, st_q = 0.0f;
    int st_n = 0;
    auto st_add = [&](float x) {
      if (st_n == 0) st_sh = x;
      const float d = x - st_sh;
      st_s += d;
      st_q = fmaf(d, d, st_q);
      ++st_n;
    };
#pragma unroll
    for (int jj = 0; jj < S::J2; ++jj) {
      const int j = t + S::R2 * jj;
      float2 u[S::R2];
      if (act2) {
        u[0] = mybuf[j];
#pragma unroll
        for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[j + S::R1P * r], cconj(tw2[j * S::R2 + r]));
      }
      if (jj == S::J2 - 1) {
        if (stage) {
          __syncthreads();  // every stage-2 input read: buf takes the output rows
        } else {
          fence_proxy_async_smem();  // this thread's accesses of buf precede the next bulk copy into it
          __syncthreads();           // buf free
          if (tid == 0 && w + (int)gridDim.x < items) issue(w + gridDim.x, false);
          if (tid == 0 && w + 2 * (int)gridDim.x < items) issue(w + 2 * gridDim.x, true);
          prefetch(w + gridDim.x);
        }
      }
      if (act2) {
        dft_reg<S::R2, +1>(u);
#pragma unroll
        for (int s2 = 0; s2 < S::R2; ++s2) {
          const int jc = j + S::R1 * s2 - kP;
          // columns of this stage inside [0, WMIN) for every t need no crop test
          const bool sure = (S::R2 * jj + S::R1 * s2 >= kP) && (S::R2 * jj + S::JSPAN - 1 + S::R1 * s2 - kP < S::WMIN);
          if (sure || (jc >= 0 && jc < A.W)) {
            const T qa = f_from_f<T>(u[s2].x - u00), qb = f_from_f<T>(u[s2].y - u00);
            if (stage) {
              srows[(size_t)(2 * f) * A.W + jc] = qa;
              srows[(size_t)(2 * f + 1) * A.W + jc] = qb;
            } else {
              if (va) o[(size_t)ia * A.W + jc] = qa;
              if (vb) o[(size_t)ib * A.W + jc] = qb;
            }
            if constexpr (STATS) {
              if (va) st_add(f_to_f(qa));
              if (vb) st_add(f_to_f(qb));
            }
          }
        }
      }
    }
    if (stage) {
      fence_proxy_async_smem();  // the staged rows precede the bulk copy that reads them
      __syncthreads();
      if (tid == 0) {
        const int r0 = g * 2 * S::F, nr = (A.H - r0) < 2 * S::F ? (A.H - r0) : 2 * S::F;
        bulk_store(o + (size_t)r0 * A.W, srows, (unsigned)((size_t)nr * A.W * sizeof(T)));
        bulk_store_wait_read();  // buf read out: the next item may land in it
        if (w + (int)gridDim.x < items) issue(w + gridDim.x, false);
        if (w + 2 * (int)gridDim.x < items) issue(w + 2 * gridDim.x, true);
      }
      prefetch(w + gridDim.x);
    }
    if constexpr (STATS) {
      // (count, mean, M2) of the thread, combined pairwise (Chan et al.'s update,
      // stable in FP32) down a shuffle tree and across the warps in order; the
      // item's (count, mean, M2) go out in FP64
      float cn = (float)st_n, cm = st_n ? st_sh + st_s / cn : 0.0f, c2 = st_n ? st_q - st_s * (st_s / cn) : 0.0f;
      auto chan = [](float& n, float& m, float& m2, float nb, float mb, float m2b) {
        const float nt = n + nb;
        if (nt > 0.0f) {
          const float d = mb - m, fb = nb / nt;
          m = fmaf(d, fb, m);
          m2 = m2 + m2b + d * d * n * fb;
        }
        n = nt;
      };
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        const float nb = __shfl_xor_sync(0xffffffffu, cn, o2), mb = __shfl_xor_sync(0xffffffffu, cm, o2),
                    m2b = __shfl_xor_sync(0xffffffffu, c2, o2);
        chan(cn, cm, c2, nb, mb, m2b);
      }
      __shared__ float st_red[3 * (S::THREADS / 32)];
      if ((tid & 31) == 0) {
        st_red[3 * (tid >> 5)] = cn;
        st_red[3 * (tid >> 5) + 1] = cm;
        st_red[3 * (tid >> 5) + 2] = c2;
      }
      __syncthreads();
      if (tid == 0) {
        float n = 0.0f, m = 0.0f, m2 = 0.0f;
        for (int k = 0; k < S::THREADS / 32; ++k) chan(n, m, m2, st_red[3 * k], st_red[3 * k + 1], st_red[3 * k + 2]);
        double* dst = reinterpret_cast<double*>(partial) + (size_t)field * (kMaxRowBlocks / 2) + kStatsOff + 3 * g;
        dst[0] = (double)n;
        dst[1] = (double)m;
        dst[2] = (double)m2;
      }
      // st_red is rewritten only after the next item's barriers
    }
  }
  if (tid == 0) bulk_store_wait();  // the last staged rows are stored before the kernel ends
}

// Colour correction of Eq. 25 for fields whose statistics the inverse row pass
// took as it stored them. k_fast_color_finish: one warp per field combines the
// items' (count, mean, M2) in FP64 in a fixed order (lane-strided, then a
// shuffle tree) into the field's mean and population standard deviation and
// writes (mean, gain = ref_std / std or 0 when std = 0, ref_mean) at
// kColorCoef of the field's scratch. k_fast_color_apply maps
// x <- (x - mean) gain + ref_mean, 16 bytes per access where the field allows.
constexpr int kColorCoef = 1200;  // float offset (past the item statistics, 3 doubles per item)

__device__ __forceinline__ void chan_d(double& n, double& m, double& m2, double nb, double mb, double m2b) {
  const double nt = n + nb;
  if (nt > 0.0) {
    const double d = mb - m, fb = nb / nt;
    m += d * fb;
    m2 += m2b + d * d * n * fb;
  }
  n = nt;
}

static __global__ void __launch_bounds__(256) k_fast_color_finish(float* __restrict__ partial, int nitems, int nf,
                                                                  const float* __restrict__ ref_mean,
                                                                  const float* __restrict__ ref_std) {
  const int field = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (field >= nf) return;
  const double* pp = reinterpret_cast<const double*>(partial) + (size_t)field * (kMaxRowBlocks / 2) + kStatsOff;
  double n = 0.0, m = 0.0, m2 = 0.0;
  for (int i = lane; i < nitems; i += 32) chan_d(n, m, m2, pp[3 * i], pp[3 * i + 1], pp[3 * i + 2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double nb = __shfl_down_sync(0xffffffffu, n, o), mb = __shfl_down_sync(0xffffffffu, m, o),
                 m2b = __shfl_down_sync(0xffffffffu, m2, o);
    chan_d(n, m, m2, nb, mb, m2b);
  }
  if (lane == 0) {
    const double sd = n > 0.0 ? sqrt(fmax(m2 / n, 0.0)) : 0.0;
    float* c = partial + (size_t)field * kMaxRowBlocks + kColorCoef;
    c[0] = (float)m;
    c[1] = sd > 0.0 ? (float)((double)ref_std[field] / sd) : 0.0f;
    c[2] = ref_mean[field];
  }
}

template <typename T, int V>
__global__ void __launch_bounds__(256) k_fast_color_apply(T* __restrict__ out, const float* __restrict__ partial,
                                                          long long n) {
  const int field = blockIdx.y;
  const float* c = partial + (size_t)field * kMaxRowBlocks + kColorCoef;
  const float mc = c[0], gsc = c[1], mi = c[2];
  T* x = out + (long long)field * n;
  const long long nv = n / V;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    if constexpr (V == 4) {
      float4 v = reinterpret_cast<float4*>(x)[i];
      v.x = fmaf(v.x - mc, gsc, mi);
      v.y = fmaf(v.y - mc, gsc, mi);
      v.z = fmaf(v.z - mc, gsc, mi);
      v.w = fmaf(v.w - mc, gsc, mi);
      reinterpret_cast<float4*>(x)[i] = v;
    } else {
      x[i] = f_from_f<T>(fmaf(f_to_f(x[i]) - mc, gsc, mi));
    }
  }
}

// ---------------------------------------------------------------------------
// adjoint pass C: w = inverse transform of the row-major spectrum Y (rows
// 0..H, torus rows p..p+H). The transpose of the divergence is formed in the
// row-frequency domain, one output row i per transform:
//   grad_gx[i] = F^-1((1 - exp(2 pi i l / N)) Y[i])     (w[i][j] - w[i][j+1])
//   grad_gy[i] = F^-1(Y[i] - Y[i+1])                   (w[i][j] - w[i+1][j])
// Both spectra are Hermitian, so one complex inverse transform of
// A + i B gives grad_gx in its real part and grad_gy in its imaginary part.
// ---------------------------------------------------------------------------
// Recursive column solve, the adjoint's inverse pass side: the F staged rows of
// half-band g of S (and row F, the next half-band's first row) become rows of
// the solved spectrum U in place, from the half-band's two carries, one column
// per thread: the causal recursion down the half-band, row F from the causal
// value above it and the anticausal carry (which is y' at row F), then the
// anticausal recursion up, U = C_l (y + y' - X). Column 0 already holds its
// exact solution; rows past the torus are left alone (no output row needs them).
template <class S>
__device__ __forceinline__ void tri_solve_half(float2* stg, const float2* cbuf, const float* __restrict__ cc, int g,
                                               const FastArgs& A) {
  constexpr int F = S::F;
  const int nb = min(F, A.M - A.p - g * F);
  const bool extra = nb == F && g * F + F < A.srows;
  const float2* dcs = reinterpret_cast<const float2*>(cc + (size_t)A.Nh * 8);  // (delta, C) per column
  for (int k = 1 + threadIdx.x; k < A.Nh; k += blockDim.x) {
    const float2 dc = __ldg(dcs + k);
    float2 yc = cbuf[k], ya = cbuf[S::LDY + k];
    float2* col = stg + k;
    float2 x[F + 1];
#pragma unroll
    for (int r = 0; r < F; ++r) x[r] = col[(size_t)r * S::LDY];
    x[F] = extra ? col[(size_t)F * S::LDY] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < F; ++r)
      if (r < nb) {
        yc = tri_step(x[r], yc, dc.x);
        col[(size_t)r * S::LDY] = yc;
      }
    if (extra) col[(size_t)F * S::LDY] = cscale(csub(cadd(tri_step(x[F], yc, dc.x), ya), x[F]), dc.y);
#pragma unroll
    for (int r = F - 1; r >= 0; --r)
      if (r < nb) {
        ya = tri_step(x[r], ya, dc.x);
        col[(size_t)r * S::LDY] = cscale(csub(cadd(col[(size_t)r * S::LDY], ya), x[r]), dc.y);
      }
  }
}

// TRI: the recursive column solve's adjoint; Y is then the row-major spectrum
// S of Crop^T(grad_out) (srows rows per field), an item is half-band g (output
// rows gF .. gF + F - 1), whose F + 1 rows of S and two carries arrive by bulk
// copy and are solved in place (tri_solve_half) before the output transforms.
template <class S, typename T, bool TRI = false>
__global__ void __launch_bounds__(S::THREADS, S::MINB_ADJ) k_fast_rows_adj(const float2* __restrict__ Y, T* __restrict__ ggx,
                                                                 T* __restrict__ ggy, const float2* __restrict__ twg,
                                                                 FastArgs A, const float2* __restrict__ tri = nullptr,
                                                                 const float* __restrict__ cc = nullptr) {
  extern __shared__ __align__(16) float2 sm[];
  float2* tw2 = sm;                          // [R1][R2]: w_N^(r j)
  float2* buf = sm + S::R1 * S::R2;          // [F][NP] exchange
  float2* dtab = buf + S::F * S::NP;         // [N/2 + 1] 1 - exp(2 pi i l / N)
  float2* stg = reinterpret_cast<float2*>(reinterpret_cast<char*>(sm) + S::adj_stage_offset());  // [F + 1][ldY]
  float2* cbuf = stg + (size_t)(S::F + 1) * S::LDY;  // TRI: the half-band's carries [2][LDY]
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int f = tid / S::T, t = tid - f * S::T;
  const bool act = f < S::F;
  const int half = S::N / 2;
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    tw2[i] = twg[r * j];
  }
  for (int l = tid; l <= half; l += blockDim.x) {
    // 1 - cos is formed as sin^2 / (1 + cos) where cos > 0, avoiding the
    // cancellation near DC; the imaginary part is -sin
    const float2 e = twg[l];
    const float cs = e.x, sn = -e.y;
    dtab[l] = make_float2((cs > 0.0f) ? __fdividef(sn * sn, 1.0f + cs) : 1.0f - cs, -sn);
  }
  float2* mybuf = buf + (act ? f : 0) * S::NP;
  const int items = A.nf * A.ngroups;
  // one thread: rows gF .. gF + F of Y (fewer at the end of a field); prefetch:
  // only start fetching them into L2, for the copy one item later
  auto issue = [&](int w, bool prefetch) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    const int r0 = g * S::F;
    if constexpr (TRI) {
      const int nr = (A.srows - r0) < S::F + 1 ? (A.srows - r0) : S::F + 1;
      const float2* ys = Y + ((size_t)field * A.srows + r0) * A.ldY;
      const float2* cs = tri + (size_t)field * A.tri_field + (size_t)g * 2 * A.ldY;
      const unsigned nb = (unsigned)(nr * A.ldY * sizeof(float2)), cb = (unsigned)(2 * A.ldY * sizeof(float2));
      if (prefetch) {
        l2_prefetch(ys, nb);
        l2_prefetch(cs, cb);
      } else {
        mbar_expect_tx(&bar, nb + cb);
        bulk_copy(stg, ys, nb, &bar);
        bulk_copy(cbuf, cs, cb, &bar);
      }
      return;
    }
    const int nr = (A.H + 1 - r0) < S::F + 1 ? (A.H + 1 - r0) : S::F + 1;
    const float2* ys = Y + ((size_t)field * (A.H + 1) + r0) * A.ldY;
    const unsigned nb = (unsigned)(nr * A.ldY * sizeof(float2));
    if (prefetch)
      l2_prefetch(ys, nb);
    else
      bulk_load(stg, ys, nb, &bar);
  };
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < items) issue(blockIdx.x, false);
  if (tid == 0 && (int)(blockIdx.x + gridDim.x) < items) issue(blockIdx.x + gridDim.x, true);
  unsigned phase = 0;
#pragma unroll 1
  for (int w = blockIdx.x; w < items; w += gridDim.x, phase ^= 1u) {
    const int field = w / A.ngroups, g = w - field * A.ngroups;
    const int i = g * S::F + f;  // output row of this transform
    const bool vi = act && i < A.H;
    const bool landed = mbar_wait(&bar, phase);
    if constexpr (TRI) {
      if (__syncthreads_or(!landed)) {  // the copies never completed: report, let them drain, stop
        if (tid == 0) atomicExch(A.err, kErrBulkWait);
        mbar_wait(&bar, phase);
        return;
      }
      tri_solve_half<S>(stg, cbuf, cc, g, A);
      __syncthreads();
    }
    const float2* y0 = stg + (size_t)(vi ? f : 0) * A.ldY;
    const float2* y1 = y0 + A.ldY;  // row i + 1 (Y holds H + 1 rows)
    float2 v[S::R1];
#pragma unroll
    for (int r = 0; r < S::R1; ++r) {
      const int l = t + S::R2 * r;
      const bool all_lo = S::R2 * r + S::R2 - 1 < half;
      const bool all_hi = S::R2 * r > half;
      const bool lo = all_lo || (!all_hi && l < half);
      const int src = lo ? l : S::N - l;
      float2 ya = vi ? y0[src] : make_float2(0.0f, 0.0f);
      float2 yb = vi ? y1[src] : make_float2(0.0f, 0.0f);
      const bool may_edge = (r == 0) || (!all_lo && !all_hi);
      if (may_edge && (src == 0 || src == half)) {
        ya.y = 0.0f;
        yb.y = 0.0f;
      }
      const float2 a = cmul(ya, dtab[src]);
      const float2 b = csub(ya, yb);
      v[r] = lo ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, b.x - a.y);
    }
    fence_proxy_async_smem();  // this thread's reads of the staged rows precede the next bulk copy
    if (__syncthreads_or(!landed)) {  // the copy never completed: report, let it drain, stop
      if (tid == 0) atomicExch(A.err, kErrBulkWait);
      mbar_wait(&bar, phase);
      return;
    }
    // every staged row read, and the previous item's stage 2 done with buf
    if (tid == 0 && w + (int)gridDim.x < items) issue(w + gridDim.x, false);
    if (tid == 0 && w + 2 * (int)gridDim.x < items) issue(w + 2 * gridDim.x, true);
    if (act) {
      dft_reg<S::R1, +1>(v);
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();
    if (act && t < S::JSPAN && vi) {
      T* ox = ggx + (size_t)field * A.H * A.W + (size_t)i * A.W;
      T* oy = ggy + (size_t)field * A.H * A.W + (size_t)i * A.W;
#pragma unroll
      for (int jj = 0; jj < S::J2; ++jj) {
        const int j = t + S::R2 * jj;
        float2 u[S::R2];
        u[0] = mybuf[j];
#pragma unroll
        for (int r = 1; r < S::R2; ++r) u[r] = cmul(mybuf[j + S::R1P * r], cconj(tw2[j * S::R2 + r]));
        dft_reg<S::R2, +1>(u);
#pragma unroll
        for (int s2 = 0; s2 < S::R2; ++s2) {
          const int jc = j + S::R1 * s2 - kP;
          const bool sure = (S::R2 * jj + S::R1 * s2 >= kP) && (S::R2 * jj + S::JSPAN - 1 + S::R1 * s2 - kP < S::WMIN);
          if (sure || (jc >= 0 && jc < A.W)) {
            ox[jc] = f_from_f<T>(u[s2].x);
            oy[jc] = f_from_f<T>(u[s2].y);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side: one size pair (row schedule RS, column schedule CS)
// ---------------------------------------------------------------------------

// Packed-row buffer elements per field: it holds pass L's packed rows and later
// pass B's row-major output (H + 1 rows for the adjoint).
template <class RS>
size_t fast_zbuf_elems_for(int H) {
  const size_t groups = (size_t)(((H + 2) / 2) + RS::F - 1) / RS::F;
  const size_t packed = groups * RS::F * ((RS::N + 3) & ~3);
  const size_t rows = (size_t)(H + 1) * (((RS::N / 2 + 1) + 3) & ~3);
  return packed > rows ? packed : rows;
}

// Bands of the recursive column solve for an H-row image (the gradient's
// row pairs grouped F at a time: pass A's items).
template <class RS>
int fast_tri_groups_for(int H) {
  return (((H + 2) / 2) + RS::F - 1) / RS::F;
}

// Set the kernel's shared-memory cap (each kernel here has one fixed size) and
// return how many blocks of it fit on the device at once.
template <typename K>
static cudaError_t fast_setup(K kernel, int threads, size_t smem, int* slots) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *slots = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

}  // namespace gfc

// the one-launch solve for small tori (thread-block clusters, spectrum kept in
// shared memory), tried first by plain gradient solves below
#include "fused_small.cuh"

namespace gfc {

// The adjoint on a plan with the recursive column solve (reading: the
// transpose of the solve, z = Crop^T(grad_out) - (sum grad_out) e_00 through
// the same Green operator, then the forward differences' transposes): the
// forward row pass packs grad_out into z's rows (row-pair sums for the e_00
// term) and stores S with half-band sums; one warp per field reduces the sum;
// the carry sweep runs over the half-bands with -sum at torus row 0; the
// adjoint's inverse row pass solves each half-band in shared memory and writes
// grad_gx, grad_gy. Needs grad_out rows that can be bulk-copied into the
// forward pass's staging; returns cudaErrorNotSupported otherwise.
template <class RS, typename T>
static cudaError_t run_fast_adj_tri(gfc_plan* P, const Bufs& bf, const T* gout, T* ggx, T* ggy, int nf,
                                    cudaStream_t st) {
  if ((P->W * sizeof(T)) % 16 != 0 || (size_t)2 * RS::F * P->W * sizeof(T) > fused_exchange_bytes<RS>() ||
      getenv("GFC_UNFUSED_DIV") != nullptr)
    return cudaErrorNotSupported;
  FastArgs A;
  A.stage_out = 0;
  A.invM = 1.0 / (double)P->M;
  A.invN = 1.0 / (double)P->N;
  A.adj = 1;
  A.l2res = 0;
  A.H = P->H; A.W = P->W; A.p = P->pad; A.M = P->M; A.N = P->N; A.Nh = P->Nh; A.ldM = P->ldM;
  A.nrows = P->H;
  A.ncols = P->W;
  A.npairs = (A.nrows + 1) / 2;
  A.ldz = (RS::N + 3) & ~3;
  A.ngroups = P->triG;  // the forward pass's items: the bands of 2F rows
  A.zpairs = A.ngroups * RS::F;
  A.nparts = 0;
  A.nf = nf;
  A.ldY = (P->Nh + 3) & ~3;
  A.err = P->dev_err;
  A.srows = 2 * A.zpairs;
  A.G = P->triGh;       // the sweep's half-bands of F rows
  A.tri_field = P->tri_field;
  const int nkb = (P->Nh + kTriCols - 1) / kTriCols;
  if ((size_t)2 * RS::F * A.ldY > (size_t)RS::F * RS::NP || A.zpairs > kAdjTotal ||
      (size_t)A.srows * A.ldY > P->spec_field || nkb > kTriCnt || P->M > kTriMaxM)
    return cudaErrorInvalidConfiguration;
  static std::mutex mu;
  static int slots_a = 0, slots_c = 0;
  cudaError_t e;
  {
    std::lock_guard<std::mutex> lock(mu);
    static bool ready = false;
    if (!ready) {
      int unused = 0;
      if ((e = fast_setup(k_fast_rows_fwd_div<RS, T, true, true>, RS::THREADS, RS::smem_bytes_fwd(), &slots_a)) !=
          cudaSuccess)
        return e;
      if ((e = fast_setup(k_fast_rows_adj<RS, T, true>, RS::THREADS, RS::smem_bytes_adj_tri(), &slots_c)) !=
          cudaSuccess)
        return e;
      if ((e = fast_setup(k_tri_carries, 32 * (kTriSeg + 1), (size_t)2 * kTriTileMaxG * kTriCols * sizeof(float2),
                          &unused)) != cudaSuccess)
        return e;
      ready = true;
    }
  }
  const bool one = P->block_items;
  auto grid_for = [one](long items, int slots) { return (int)((one || items < slots) ? items : slots); };
  prof_begin(P, 0, st);
  k_fast_rows_fwd_div<RS, T, true, true><<<grid_for((long)nf * A.ngroups, slots_a), RS::THREADS,
                                           RS::smem_bytes_fwd(), st>>>(gout, nullptr, bf.spec, P->twN, bf.partial, A,
                                                                       bf.tri, P->colcoef_h);
  prof_end(P, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  prof_begin(P, 1, st);
  double* pd = reinterpret_cast<double*>(bf.partial);
  k_adj_total<<<nf, 32, 0, st>>>(pd, A.zpairs);
  P->prof.launches[1] += 1;  // a second launch in this pass
  if (A.G <= kTriRegG && (size_t)kTriRegWarps * (P->M + 4) * sizeof(float) <= 48 * 1024) {
    const int tasks = nf * nkb;
    k_tri_carries_reg<<<(tasks + kTriRegWarps - 1) / kTriRegWarps, 32 * kTriRegWarps,
                        (size_t)kTriRegWarps * (P->M + 4) * sizeof(float), st>>>(bf.spec, bf.tri, P->colcoef_h, pd, A,
                                                                                nkb);
  } else {
    const size_t tsm = A.G <= kTriTileMaxG ? (size_t)2 * A.G * kTriCols * sizeof(float2) : 0;
    k_tri_carries<<<dim3(nkb, nf), 32 * (kTriSeg + 1), tsm, st>>>(bf.spec, bf.tri, P->colcoef_h, P->powc_h, pd, A);
  }
  prof_end(P, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  FastArgs C = A;
  C.ngroups = (P->H + RS::F - 1) / RS::F;  // half-bands holding output rows
  prof_begin(P, 2, st);
  k_fast_rows_adj<RS, T, true><<<grid_for((long)nf * C.ngroups, slots_c), RS::THREADS, RS::smem_bytes_adj_tri(),
                                 st>>>(bf.spec, ggx, ggy, P->twN, C, bf.tri, P->colcoef_h);
  prof_end(P, st);
  return cudaGetLastError();
}

// MODE 0: solve from gradient, 1: from Laplacian, 2: adjoint (in0 = grad_out,
// out0 = grad_gx, out1 = grad_gy). Solves (modes 0 and 1) on a plan with the
// recursive column solve run pass A, the carry sweep and pass C; otherwise
// pass A, the column transforms (pass B) and pass C.
template <class RS, class CS, typename T, int MODE>
static cudaError_t run_fast_mode(gfc_plan* P, const Bufs& bf, const T* in0, const T* in1, T* out0, T* out1, int nf,
                                 cudaStream_t st, const EditArgs* ed = nullptr) {
  constexpr bool kCols = !std::is_same_v<CS, NoCols>;  // column transforms compiled for this shape
  static_assert(!kCols || RS::N <= 2048, "the adjoint packing pass covers a whole row in one block");
  if constexpr (MODE == 0) {
    if (P->tri && ed == nullptr) {  // plain solves of fields whose spectrum fits a cluster's shared memory
      const cudaError_t ef = run_fused_small<RS, T>(P, in0, in1, out0, nf, st);
      if (ef != cudaErrorNotSupported) return ef;
    }
  }
  if constexpr (MODE == 2) {
    if (P->tri) {  // the adjoint by the recursive column solve where its staging fits
      const cudaError_t ea = run_fast_adj_tri<RS, T>(P, bf, in0, out0, out1, nf, st);
      if (ea != cudaErrorNotSupported || !kCols) return ea;
    }
  }
  constexpr bool kTriMode = MODE != 2;
  const bool tri = kTriMode && P->tri;
  if (!kCols && !tri) return cudaErrorNotSupported;
  FastArgs A;
  A.stage_out = 0;
  A.invM = 1.0 / (double)P->M;
  A.invN = 1.0 / (double)P->N;
  A.adj = 0;
  A.l2res = (tri && P->l2res) ? 1 : 0;
  A.H = P->H; A.W = P->W; A.p = P->pad; A.M = P->M; A.N = P->N; A.Nh = P->Nh; A.ldM = P->ldM;
  A.nrows = (MODE == 0) ? P->H + 1 : P->H;
  A.ncols = (MODE == 0) ? P->W + 1 : P->W;
  A.npairs = (A.nrows + 1) / 2;
  A.ldz = (RS::N + 3) & ~3;
  A.ngroups = (A.npairs + RS::F - 1) / RS::F;
  if (tri) A.ngroups = P->triG;  // the bands of the column solve: every mode uses the gradient's
  A.zpairs = A.ngroups * RS::F;
  A.nparts = kCols ? (P->Nh + CS::C - 1) / CS::C : 0;
  A.nf = nf;
  A.ldY = (P->Nh + 3) & ~3;
  A.err = P->dev_err;
  A.srows = 2 * A.zpairs;
  A.G = P->triG;
  A.tri_field = P->tri_field;
  // the row passes stage their F packed rows / 2F rows of Y in the exchange buffer
  if ((size_t)2 * RS::F * A.ldY > (size_t)RS::F * RS::NP || A.ldz > RS::NP || A.zpairs > kAdjTotal)
    return cudaErrorInvalidConfiguration;
  if (tri && (size_t)A.srows * A.ldY > P->spec_field) return cudaErrorInvalidConfiguration;
  if (tri && (P->Nh + kTriCols - 1) / kTriCols > kTriCnt) return cudaErrorInvalidConfiguration;
  static std::mutex mu;
  static int slots_a = 0, slots_b = 0, slots_c = 0, slots_d = 0, slots_ta = 0, slots_tc = 0, slots_td = 0,
             slots_ts = 0, slots_tde = 0;
  cudaError_t e;
  {
    std::lock_guard<std::mutex> lock(mu);
    static bool ready = false;
    if (!ready) {
      int unused = 0;
      if ((e = fast_setup(k_fast_div<T, MODE>, 512, 0, &unused)) != cudaSuccess) return e;
      if constexpr (kCols) {
        if ((e = fast_setup(k_fast_cols<CS, MODE>, CS::THREADS, CS::smem_bytes(), &slots_b)) != cudaSuccess) return e;
        if constexpr (MODE == 2) {
          if ((e = fast_setup(k_fast_rows_adj<RS, T>, RS::THREADS, RS::smem_bytes_adj(), &slots_c)) != cudaSuccess)
            return e;
        } else {
          if ((e = fast_setup(k_fast_rows_inv<RS, T, false, false>, RS::THREADS, RS::smem_bytes(), &slots_c)) !=
              cudaSuccess)
            return e;
        }
        if ((e = fast_setup(k_fast_rows_fwd<RS, false>, RS::THREADS, RS::smem_bytes_fwd(), &slots_a)) != cudaSuccess)
          return e;
        if (MODE != 1 && (e = fast_setup(k_fast_rows_fwd_div<RS, T, MODE == 2, false>, RS::THREADS,
                                         RS::smem_bytes_fwd(), &slots_d)) != cudaSuccess)
          return e;
      }
      if constexpr (MODE != 2) {
        int unused_k = 0;
        if ((e = fast_setup(k_tri_carries, 32 * (kTriSeg + 1), (size_t)2 * kTriTileMaxG * kTriCols * sizeof(float2),
                            &unused_k)) != cudaSuccess)
          return e;
        if ((e = fast_setup(k_fast_rows_inv<RS, T, true, false>, RS::THREADS, RS::smem_bytes_tri_inv(), &slots_tc)) !=
            cudaSuccess)
          return e;
        if ((e = fast_setup(k_fast_rows_fwd<RS, true>, RS::THREADS, RS::smem_bytes_fwd(), &slots_ta)) != cudaSuccess)
          return e;
      }
      if constexpr (MODE == 0) {
        if ((e = fast_setup(k_fast_rows_inv<RS, T, true, true>, RS::THREADS, RS::smem_bytes_tri_inv(), &slots_ts)) !=
            cudaSuccess)
          return e;
        if ((e = fast_setup(k_fast_rows_fwd_div<RS, T, false, true>, RS::THREADS, RS::smem_bytes_fwd(), &slots_td)) !=
            cudaSuccess)
          return e;
        if ((e = fast_setup(k_fast_rows_fwd_div<RS, T, false, true, kEditThreshold>, RS::THREADS,
                            RS::smem_bytes_fwd(), &slots_tde)) != cudaSuccess)
          return e;
      }
      ready = true;
    }
  }
  // persistent grids (as many blocks as fit, each looping over items), or one block per item
  const bool one = P->block_items;
  auto grid_for = [one](long items, int slots) { return (int)((one || items < slots) ? items : slots); };
  // Plain gradient solves fold pass L into the row pass, and the adjoint folds
  // its packing of grad_out (with the row-pair sums) into it, when the rows can
  // be bulk-copied and their staging fits the exchange buffers.
  const size_t stage = (MODE == 2) ? (size_t)2 * RS::F * P->W * sizeof(T) : fused_stage_bytes<RS, T>(P->W);
  const int edit_kind = (MODE == 0 && ed) ? ed->kind : kEditNone;
  // the threshold edit is staged with the gradient (recursive column solve plans)
  const bool fused_edit = edit_kind == kEditThreshold && tri;
  const bool fused_div = MODE != 1 && (edit_kind == kEditNone || fused_edit) && (P->W * sizeof(T)) % 16 == 0 &&
                         stage <= fused_exchange_bytes<RS>() && getenv("GFC_UNFUSED_DIV") == nullptr;
  const long a_items = (long)nf * A.ngroups;
  if (fused_div) {
    prof_begin(P, 0, st);
    if constexpr (MODE == 0) {
      if (fused_edit)
        k_fast_rows_fwd_div<RS, T, false, true, kEditThreshold>
            <<<grid_for(a_items, slots_tde), RS::THREADS, RS::smem_bytes_fwd(), st>>>(
                in0, in1, bf.spec, P->twN, bf.partial, A, bf.tri, P->colcoef, ed->t2);
      else if (tri)
        k_fast_rows_fwd_div<RS, T, false, true><<<grid_for(a_items, slots_td), RS::THREADS, RS::smem_bytes_fwd(), st>>>(
            in0, in1, bf.spec, P->twN, bf.partial, A, bf.tri, P->colcoef);
      else if constexpr (kCols)
        k_fast_rows_fwd_div<RS, T, false, false><<<grid_for(a_items, slots_d), RS::THREADS, RS::smem_bytes_fwd(), st>>>(
            in0, in1, bf.spec, P->twN, bf.partial, A, nullptr, nullptr);
    } else if constexpr (kCols) {
      k_fast_rows_fwd_div<RS, T, MODE == 2, false><<<grid_for(a_items, slots_d), RS::THREADS, RS::smem_bytes_fwd(), st>>>(
          in0, in1, bf.spec, P->twN, bf.partial, A, nullptr, nullptr);
    }
    prof_end(P, st);
  }
  if (!fused_div) prof_begin(P, 3, st);
  {
    const int nq = A.ldz / 4;
    const int bx = (MODE == 2) ? ((nq + 31) / 32) * 32 : (nq >= 256 ? 256 : ((nq + 31) / 32) * 32);
    const dim3 grid((nq + bx - 1) / bx, A.zpairs, nf);
    const int kind = fused_div ? kEditNone : edit_kind;  // a fused edit needs no pass L
    const int ex = ((nq + 31) / 32) * 32 <= 512 ? ((nq + 31) / 32) * 32 : 256;  // whole warps
    const dim3 egrid((nq + ex - 1) / ex, (A.zpairs + kEditPairs - 1) / kEditPairs, nf);
    if (kind == kEditThreshold)
      k_fast_div_edit<T, kEditThreshold><<<egrid, ex, 0, st>>>(in0, in1, nullptr, ed->t2, 0.0f, bf.zbuf, A);
    else if (kind == kEditMerge)
      k_fast_div_edit<T, kEditMerge><<<egrid, ex, 0, st>>>(in0, in1, static_cast<const T*>(ed->edges), nullptr,
                                                           ed->alpha, bf.zbuf, A);
    else if (!fused_div)
      k_fast_div<T, MODE><<<grid, bx, 0, st>>>(in0, in1, bf.zbuf, bf.partial, A);
  }
  if (!fused_div) {
    prof_end(P, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_begin(P, 0, st);
    if (tri)
      k_fast_rows_fwd<RS, true><<<grid_for(a_items, slots_ta), RS::THREADS, RS::smem_bytes_fwd(), st>>>(
          bf.zbuf, bf.spec, P->twN, A, bf.tri, P->colcoef, bf.partial);
    else if constexpr (kCols)
      k_fast_rows_fwd<RS, false><<<grid_for(a_items, slots_a), RS::THREADS, RS::smem_bytes_fwd(), st>>>(
          bf.zbuf, bf.spec, P->twN, A, nullptr, nullptr);
    prof_end(P, st);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  prof_begin(P, 1, st);
  const int nkb = (P->Nh + kTriCols - 1) / kTriCols;  // column blocks of the sweep (u[0,0] partials)
  if (tri && A.G <= kTriRegG && (size_t)kTriRegWarps * (P->M + 4) * sizeof(float) <= 48 * 1024) {
    const int tasks = nf * nkb;
    k_tri_carries_reg<<<(tasks + kTriRegWarps - 1) / kTriRegWarps, 32 * kTriRegWarps,
                        (size_t)kTriRegWarps * (P->M + 4) * sizeof(float), st>>>(
        bf.spec, bf.tri, P->colcoef, reinterpret_cast<double*>(bf.partial), A, nkb);
  } else if (tri) {
    const size_t tsm = A.G <= kTriTileMaxG ? (size_t)2 * A.G * kTriCols * sizeof(float2) : 0;
    k_tri_carries<<<dim3(nkb, nf), 32 * (kTriSeg + 1), tsm, st>>>(bf.spec, bf.tri, P->colcoef, P->powc,
                                                                   reinterpret_cast<double*>(bf.partial), A);
  } else if constexpr (kCols) {
    if (MODE == 2) {
      k_adj_total<<<nf, 32, 0, st>>>(reinterpret_cast<double*>(bf.partial), A.zpairs);
      P->prof.launches[1] += 1;  // a second launch in this pass
    }
    k_fast_cols<CS, MODE><<<grid_for((long)nf * A.nparts, slots_b), CS::THREADS, CS::smem_bytes(), st>>>(
        bf.spec, bf.zbuf, P->GT, P->twM, bf.partial, A);
  }
  prof_end(P, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  FastArgs C = A;
  // the inverse row pass stages its output rows in its exchange buffer and
  // stores them by bulk copy when the rows are whole 16-byte multiples
  C.stage_out = MODE != 2 && (P->W * sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(out0) & 15) == 0 &&
                (size_t)2 * RS::F * P->W * sizeof(T) <= (size_t)RS::F * RS::NP * sizeof(float2);
  prof_begin(P, 2, st);
  if constexpr (MODE == 2) {
    C.ngroups = (P->H + RS::F - 1) / RS::F;
    k_fast_rows_adj<RS, T><<<grid_for((long)nf * C.ngroups, slots_c), RS::THREADS, RS::smem_bytes_adj(), st>>>(
        bf.zbuf, out0, out1, P->twN, C);
  } else {
    (void)out1;
    C.ngroups = ((P->H + 1) / 2 + RS::F - 1) / RS::F;
    const bool stats = MODE == 0 && tri && ed && ed->ref_mean;
    if (stats && (kStatsOff + 3 * C.ngroups > kColorCoef / 2 || nkb > kStatsOff)) return cudaErrorInvalidConfiguration;
    if (stats) {
      C.nparts = nkb;
      k_fast_rows_inv<RS, T, true, true>
          <<<grid_for((long)nf * C.ngroups, slots_ts), RS::THREADS, RS::smem_bytes_tri_inv(), st>>>(
              bf.spec, bf.partial, out0, P->twN, C, bf.tri, P->colcoef);
    } else if (tri) {
      C.nparts = nkb;
      k_fast_rows_inv<RS, T, true, false>
          <<<grid_for((long)nf * C.ngroups, slots_tc), RS::THREADS, RS::smem_bytes_tri_inv(), st>>>(
              bf.spec, bf.partial, out0, P->twN, C, bf.tri, P->colcoef);
    } else if constexpr (kCols) {
      k_fast_rows_inv<RS, T, false, false>
          <<<grid_for((long)nf * C.ngroups, slots_c), RS::THREADS, RS::smem_bytes(), st>>>(
              bf.zbuf, bf.partial, out0, P->twN, C, nullptr, nullptr);
    }
    if (stats) {
      prof_end(P, st);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      prof_begin(P, 3, st);  // counted with the other non-transform pass
      const long long n = (long long)P->H * P->W;
      k_fast_color_finish<<<(nf + 7) / 8, 256, 0, st>>>(bf.partial, C.ngroups, nf, ed->ref_mean, ed->ref_std);
      const bool v4 = sizeof(T) == 4 && n % 4 == 0 && (reinterpret_cast<uintptr_t>(out0) & 15) == 0;
      const long long per = v4 ? n / 4 : n;
      int nblk = (int)((per + 256 * 8 - 1) / (256 * 8));
      if (nblk < 1) nblk = 1;
      if (v4)
        k_fast_color_apply<T, 4><<<dim3(nblk, nf), 256, 0, st>>>(out0, bf.partial, n);
      else
        k_fast_color_apply<T, 1><<<dim3(nblk, nf), 256, 0, st>>>(out0, bf.partial, n);
    }
  }
  prof_end(P, st);
  return cudaGetLastError();
}

// Shapes compiled for their row length only (the recursive column solve needs
// no column kernels): FP32 solves and edited solves; the caller falls back to
// the generic passes for anything else (cudaErrorNotSupported).
template <class RS>
cudaError_t run_rows_shape(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                           void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  if (P->dtype != GFC_F32 || !P->tri) return cudaErrorNotSupported;
  const float* a = static_cast<const float*>(in0);
  const float* b = static_cast<const float*>(in1);
  float* o0 = static_cast<float*>(out0);
  float* o1 = static_cast<float*>(out1);
  if (mode == 0) return run_fast_mode<RS, NoCols, float, 0>(P, bf, a, b, o0, o1, nf, st, ed);
  if (mode == 2) return run_fast_mode<RS, NoCols, float, 2>(P, bf, a, b, o0, o1, nf, st);
  return run_fast_mode<RS, NoCols, float, 1>(P, bf, a, b, o0, o1, nf, st);
}

template <class RS, class CS>
cudaError_t run_fast_shape(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                           void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  auto go = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    const T* a = static_cast<const T*>(in0);
    const T* b = static_cast<const T*>(in1);
    T* o0 = static_cast<T*>(out0);
    T* o1 = static_cast<T*>(out1);
    if (mode == 0) return run_fast_mode<RS, CS, T, 0>(P, bf, a, b, o0, o1, nf, st, ed);
    if (mode == 1) return run_fast_mode<RS, CS, T, 1>(P, bf, a, b, o0, o1, nf, st);
    return run_fast_mode<RS, CS, T, 2>(P, bf, a, b, o0, o1, nf, st);
  };
  switch (P->dtype) {
    case GFC_F32: return go(float{});
    case GFC_F16: return go(__half{});
    default: return go(__nv_bfloat16{});
  }
}

}  // namespace gfc

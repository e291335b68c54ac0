// fused_small.cuh -- one-launch solve from gradients for small tori.
//
// The three steps of the recursive column solve (row transforms with band
// sums, the carry sweep, the in-band solve with the inverse row transforms;
// Eq. 23's Green multiply applied as the inverse of the cyclic tridiagonal
// operator along the torus rows, Algorithm B's offset and crop) run in one
// kernel: a thread-block cluster per field, each CTA owning a contiguous run
// of bands of 2F torus rows. A CTA keeps its bands of the row-major spectrum S
// in its own shared memory from the row transforms to the inverse ones, so S
// never goes to HBM; the only data that cross CTAs are the bands' causal and
// anticausal sums and column 0 of S, read through distributed shared memory
// between two cluster barriers. Each CTA folds every band's sums (the same
// fold, in the same order, in every CTA of the cluster) to get the carries into
// and below its own bands and u[0,0]; warp 0 solves column 0 exactly in FP64.
// gx and gy are read once and out written once: the minimum bytes of the path.
// It applies where a field's spectrum fits the shared memory of a cluster of
// at most eight CTAs (short rows); by default it is taken for latency-bound
// launches of tori of at most 8 bands (one band per CTA: 72 x 108 and the like).
#pragma once

#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <utility>

#include "fast_kernels.cuh"

namespace gfc {

constexpr int kFusedMaxCluster = 8;                   // portable cluster size
constexpr int kFusedMaxTiles = 40;                    // 32-column tiles of the half spectrum (N <= 2558)
constexpr size_t kFusedSmemTwoPerSM = 113 * 1024;     // two CTAs per SM
constexpr size_t kFusedSmemMax = 225 * 1024;          // one CTA per SM (with the kernel's static shared memory)

// Shared-memory carve-up of one CTA with gc bands (float2 units, every part a
// multiple of 16 bytes): twiddles [R1 R2]; the exchange buffers (staging of
// the band's gradient rows, then the stage-1 exchange [F][NP] and the stage-2
// output [F][NO]); S of the CTA's bands [gc][2F][LDY]; their sums
// [gc][2][LDY] (causal, anticausal); their carries [gc][2][LDY] (into the band,
// from below it); column 0's solution [srows]; column 0 of every S row as
// floats [M + 4].
template <class S, typename T>
struct FusedSmall {
  static constexpr int RW = 2 * S::F;
  __host__ __device__ static constexpr size_t al2(size_t n) { return (n + 1) & ~(size_t)1; }
  __host__ __device__ static constexpr size_t xbuf_elems(int W) {
    const size_t ex = (size_t)S::F * S::NP + (size_t)S::F * S::NO;
    const size_t st = (fused_stage_bytes<S, T>(W) + sizeof(float2) - 1) / sizeof(float2);
    return ex > st ? ex : st;
  }
  __host__ __device__ static constexpr size_t off_x() { return al2((size_t)S::R1 * S::R2); }
  __host__ __device__ static constexpr size_t off_s(int W) { return off_x() + al2(xbuf_elems(W)); }
  __host__ __device__ static constexpr size_t off_sum(int W, int gc) {
    return off_s(W) + (size_t)gc * RW * S::LDY;
  }
  __host__ __device__ static constexpr size_t off_car(int W, int gc) {
    return off_sum(W, gc) + (size_t)gc * 2 * S::LDY;
  }
  __host__ __device__ static constexpr size_t off_c0(int W, int gc) {
    return off_car(W, gc) + (size_t)gc * 2 * S::LDY;
  }
  __host__ __device__ static constexpr size_t off_fcol(int W, int gc, int srows) {
    return off_c0(W, gc) + al2((size_t)srows);
  }
  __host__ __device__ static constexpr size_t bytes(int W, int gc, int srows, int M) {
    return (off_fcol(W, gc, srows) + al2(((size_t)M + 5) / 2)) * sizeof(float2);
  }
};

// first band of CTA c of a cluster of cl CTAs over G bands (every CTA gets
// floor or ceil of G / cl bands; cl <= G, so none is empty)
__device__ __forceinline__ int fused_band0(int c, int G, int cl) { return (int)(((long)c * G) / cl); }
__device__ __forceinline__ int fused_owner(int g, int G, int cl) {
  int c = 0;
  while (fused_band0(c + 1, G, cl) <= g) ++c;
  return c;
}

template <class S, typename T>
__global__ void __launch_bounds__(S::THREADS, 2) k_fused_small(const T* __restrict__ gx, const T* __restrict__ gy,
                                                               T* __restrict__ out, const float2* __restrict__ twg,
                                                               const float* __restrict__ cc, FastArgs A, int cl,
                                                               int gc) {
  namespace cg = cooperative_groups;
  using L = FusedSmall<S, T>;
  constexpr int RW = L::RW;
  constexpr int LDY = S::LDY;
  extern __shared__ __align__(16) float2 sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int field = (int)(blockIdx.x / (unsigned)cl);
  float2* tw2 = sm;
  float2* xbuf = sm + L::off_x();
  float2* buf2 = xbuf + S::F * S::NP;
  float2* sres = sm + L::off_s(A.W);
  float2* sums = sm + L::off_sum(A.W, gc);
  float2* car = sm + L::off_car(A.W, gc);
  float2* col0 = sm + L::off_c0(A.W, gc);
  float* fcol = reinterpret_cast<float*>(sm + L::off_fcol(A.W, gc, A.srows));
  __shared__ __align__(8) uint64_t bar;
  __shared__ double tile_u[kFusedMaxTiles];  // u[0,0] partial of each 32-column tile
  __shared__ float u00s;
  __shared__ unsigned char bown[kTriRegG], bloc[kTriRegG];  // owner CTA and its local index of every band
  const int tid = threadIdx.x;
  const int f = tid / S::T, t = tid - f * S::T;
  const bool act = f < S::F;
  const int G = A.G;
  const int gb0 = fused_band0(rank, G, cl), gb1 = fused_band0(rank + 1, G, cl);
  const size_t fe = (size_t)A.H * A.W;
  T* sgx = reinterpret_cast<T*>(xbuf);  // gx rows r0 .. r0 + RW - 1
  T* sgy = sgx + (size_t)RW * A.W;      // gy rows r0 - 1 .. r0 + RW - 1
  const unsigned row = (unsigned)(A.W * sizeof(T));
  // one thread: the gradient rows of band g into the staging area
  auto issue = [&](int g) {
    const int r0 = g * RW;
    const int nx = (A.H - r0) < RW ? (A.H - r0) : RW;                            // may be 0
    const int y0 = r0 > 0 ? r0 - 1 : 0, y1 = (A.H < r0 + RW) ? A.H : r0 + RW;  // at least one row
    const T* xs = gx + field * fe + (size_t)r0 * A.W;
    const T* ys = gy + field * fe + (size_t)y0 * A.W;
    mbar_expect_tx(&bar, (unsigned)(nx > 0 ? nx : 0) * row + (unsigned)(y1 - y0) * row);
    if (nx > 0) bulk_copy(sgx, xs, (unsigned)nx * row, &bar);
    bulk_copy(sgy + (size_t)(y0 - (r0 - 1)) * A.W, ys, (unsigned)(y1 - y0) * row, &bar);
  };
  if (tid == 0) mbar_init(&bar, 1);
  if (tid < G) {
    const int o = fused_owner(tid, G, cl);
    bown[tid] = (unsigned char)o;
    bloc[tid] = (unsigned char)(tid - fused_band0(o, G, cl));
  }
  __syncthreads();
  if (tid == 0) issue(gb0);
  for (int i = tid; i < S::R1 * S::R2; i += blockDim.x) {
    const int j = i / S::R2, r = i - j * S::R2;
    tw2[i] = twg[r * j];
  }
  float2* mybuf = xbuf + (act ? f : 0) * S::NP;
  float2* mybuf2 = buf2 + (act ? f : 0) * S::NO;
  bool ok = true;
  unsigned phase = 0;
  // ---- step 1: divergence, forward row transforms, S rows and band sums
#pragma unroll 1
  for (int g = gb0; g < gb1; ++g, phase ^= 1u) {
    const int gl = g - gb0;
    const bool landed = ok ? mbar_wait(&bar, phase) : false;
    if (__syncthreads_or(!landed)) {  // the copies never completed: report, let them drain, compute no more
      if (ok) {
        if (tid == 0) atomicExch(A.err, kErrBulkWait);
        mbar_wait(&bar, phase);
      }
      ok = false;
      continue;
    }
    float2 v[S::R1];
    if (act) {
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
    __syncthreads();  // every staged row read: the staging becomes the exchange
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
    // the band's 2F rows of S (two-for-one split) and its sums with zero carries
    const int nb = min(RW, A.M - A.p - g * RW);
    float2* Sr = sres + (size_t)gl * RW * LDY;
    for (int k = tid; k < A.Nh; k += blockDim.x) {
      const int km = k == 0 ? 0 : S::N - k;
      float2 x[RW];
#pragma unroll
      for (int q = 0; q < S::F; ++q) {
        const float2 zk = buf2[q * S::NO + k], zm = buf2[q * S::NO + km];
        const float2 zc = make_float2(zm.x, -zm.y);
        x[2 * q] = cscale(cadd(zk, zc), 0.5f);
        const float2 d = csub(zk, zc);
        x[2 * q + 1] = cscale(make_float2(d.y, -d.x), 0.5f);
      }
#pragma unroll
      for (int r = 0; r < RW; ++r) Sr[(size_t)r * LDY + k] = x[r];
      const float dl = __ldg(cc + (size_t)k * 8);
      float2 e = make_float2(0.0f, 0.0f), ep = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int r = 0; r < RW; ++r)
        if (r < nb) e = tri_step(x[r], e, dl);
#pragma unroll
      for (int r = RW - 1; r >= 0; --r)
        if (r < nb) ep = tri_step(x[r], ep, dl);
      sums[(size_t)(2 * gl) * LDY + k] = e;
      sums[(size_t)(2 * gl + 1) * LDY + k] = ep;
    }
    fence_proxy_async_smem();  // this thread's accesses of the staging precede the next bulk copy
    __syncthreads();
    if (tid == 0 && g + 1 < gb1) issue(g + 1);
  }
  // ---- step 2: carries of the CTA's bands and u[0,0], from every band's sums
  cluster.sync();  // every CTA's S rows and sums are written (release / acquire across the cluster)
  // One warp per tile of 32 columns (the sweep kernel's tiles), one column per
  // lane. The carries follow the sweep's own recurrences in its order (a fold
  // of all the bands from a zero carry closes the cycle, then the carries are
  // rebuilt band by band from the top), and u[0,0] is summed per tile and
  // across tiles in the sweep's order: the result does not depend on how the
  // bands are split over the cluster, and equals the three-launch path's.
  const int lane = tid & 31, warp = tid >> 5;
  const int nkb = (A.Nh + kTriCols - 1) / kTriCols;
  for (int kb = warp; kb < nkb; kb += S::THREADS / 32) {
    const int k = kb * kTriCols + lane;
    const bool col_ok = k >= 1 && k < A.Nh;
    double acc = 0.0;
    if (col_ok) {
      const float4 c03 = __ldg(reinterpret_cast<const float4*>(cc + (size_t)k * 8));
      const float4 c47 = __ldg(reinterpret_cast<const float4*>(cc + (size_t)k * 8) + 1);
      const float a = c03.y, C = c03.z, Tb = c03.w, Tl = c47.x, Tp = c47.y, inv = c47.z, Tt = c47.w;
      // every band's sums in registers (one round of loads from the CTAs that
      // own them), then the sweep kernel's recurrences
      float2 e[kTriRegG], ep[kTriRegG];
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) {
          const float2* ps = cluster.map_shared_rank(sums, (int)bown[g]) + (size_t)(2 * bloc[g]) * LDY + k;
          e[g] = ps[0];
          ep[g] = ps[LDY];
        }
      float2 tt = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          tt = __ffma2_rn(make_float2(T, T), tt, e[g]);
        }
      const float2 yl = make_float2(Tt * tt.x * inv, Tt * tt.y * inv);  // y[M-1]
      float2 cin = make_float2(Tp * yl.x, Tp * yl.y);                   // carry into band 0
#pragma unroll
      for (int g = 0; g < kTriRegG; ++g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          if (g >= gb0 && g < gb1) car[(size_t)(2 * (g - gb0)) * LDY + k] = cin;
          cin = __ffma2_rn(make_float2(T, T), cin, e[g]);
        }
      float2 q = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int g = kTriRegG - 1; g >= 0; --g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          q = __ffma2_rn(make_float2(T, T), q, ep[g]);
        }
      const float2 y0 = make_float2(Tp * q.x * inv, Tp * q.y * inv);  // y'[0]
      float2 cbl = make_float2(Tt * y0.x, Tt * y0.y);                 // carry from below the last band
#pragma unroll
      for (int g = kTriRegG - 1; g >= 0; --g)
        if (g < G) {
          const float T = (g == G - 1) ? Tl : Tb;
          if (g >= gb0 && g < gb1) car[(size_t)(2 * (g - gb0) + 1) * LDY + k] = cbl;
          cbl = __ffma2_rn(make_float2(T, T), cbl, ep[g]);
        }
      // this column's share of u[0,0] = sum_l w_l U[0][l] (row 0 lies in the pad)
      acc = (2 * k == A.N ? 1.0 : 2.0) * (double)(C * fmaf(a, yl.x, y0.x));
    }
    acc = warp_sum_d(acc);
    if (lane == 0) tile_u[kb] = acc;
  }
  const int nr = min(A.srows, A.M - A.p);  // S rows on the torus
  if (tid < 32) {
    // column 0 of every S row (real parts), from the CTAs that own them
    for (int r = tid; r < A.M; r += 32) {
      const int i = r - A.p;
      if (i >= 0 && i < nr) {
        const int o = fused_owner(i / RW, G, cl);
        const float2* so = cluster.map_shared_rank(sres, o);
        fcol[r] = so[(size_t)(i - fused_band0(o, G, cl) * RW) * LDY].x;
      }
    }
    __syncwarp();
    FastArgs A1 = A;
    A1.ldY = 1;  // the solution goes to col0[i], i < nr
    tri_column0(col0, fcol, 0, A1, 0.0f);
  }
  __syncthreads();  // tile_u complete
  if (tid < 32) {
    // u[0,0] from the tiles' partials: lane-strided, then a fixed shuffle tree
    double s2 = 0.0;
    for (int i = tid; i < nkb; i += 32) s2 += tile_u[i];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o2);
    if (tid == 0) u00s = (float)s2;
  }
  cluster.sync();  // every read of another CTA's shared memory is done
  // column 0 of this CTA's S rows takes its exact solution
  for (int i = gb0 * RW + tid; i < gb1 * RW && i < nr; i += blockDim.x) sres[(size_t)(i - gb0 * RW) * LDY] = col0[i];
  __syncthreads();
  // ---- step 3: in-band solve, inverse row transforms, offset, crop, cast
  const float u00 = u00s;
  const int half = S::N / 2;
  T* o = out + (size_t)field * fe;
#pragma unroll 1
  for (int g = gb0; g < gb1; ++g) {
    if (g * RW >= A.H) break;  // no output rows here or below (the same for every thread)
    const int gl = g - gb0;
    float2* band = sres + (size_t)gl * RW * LDY;
    tri_solve_band<S>(band, car + (size_t)gl * 2 * LDY, cc, g, A);
    __syncthreads();  // the band's solved rows visible; the exchange is free
    const int ia = g * RW + 2 * f, ib = ia + 1;
    const bool va = act && ia < A.H, vb = act && ib < A.H;
    const float2* ya_row = band + (size_t)(va ? 2 * f : 0) * LDY;
    const float2* yb_row = band + (size_t)(vb ? 2 * f + 1 : 0) * LDY;
    float2 v[S::R1];
#pragma unroll
    for (int r = 0; r < S::R1; ++r) {
      // Hermitian extension of the two rows' half spectra, packed into one
      // complex transform (row ia real part, row ib imaginary part)
      const int l = t + S::R2 * r;
      const bool all_lo = S::R2 * r + S::R2 - 1 < half;
      const bool all_hi = S::R2 * r > half;
      const bool lo = all_lo || (!all_hi && l < half);
      const int src = lo ? l : S::N - l;
      float2 ya = va ? ya_row[src] : make_float2(0.0f, 0.0f);
      float2 yb = vb ? yb_row[src] : make_float2(0.0f, 0.0f);
      const bool may_edge = (r == 0) || (!all_lo && !all_hi);
      if (may_edge && (src == 0 || src == half)) {  // bins 0 and N/2 are real
        ya.y = 0.0f;
        yb.y = 0.0f;
      }
      v[r] = lo ? make_float2(ya.x - yb.y, ya.y + yb.x) : make_float2(ya.x + yb.y, yb.x - ya.y);
    }
    if (act) {
      dft_reg<S::R1, +1>(v);
#pragma unroll
      for (int s2 = 0; s2 < S::R1; ++s2) mybuf[t * S::R1P + s2] = v[s2];
    }
    __syncthreads();
    const bool act2 = act && t < S::JSPAN;
#pragma unroll
    for (int jj = 0; jj < S::J2; ++jj) {
      if (!act2) break;
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
          if (va) o[(size_t)ia * A.W + jc] = f_from_f<T>(u[s2].x - u00);
          if (vb) o[(size_t)ib * A.W + jc] = f_from_f<T>(u[s2].y - u00);
        }
      }
    }
  }
}

// Cluster size and bands per CTA for a plan, or 0 where the fused solve does
// not apply: the smallest cluster whose CTAs fit two per SM, else eight CTAs
// at one per SM; with few fields, clusters of up to eight CTAs so that the
// launch covers the SMs.
template <class RS, typename T>
static int fused_small_cluster(const gfc_plan* P, int nf, int sms, int* gc_out, size_t* smem_out) {
  using L = FusedSmall<RS, T>;
  const int G = P->triG, srows = 2 * G * RS::F;
  if ((P->W * sizeof(T)) % 16 != 0 || (P->Nh + kTriCols - 1) / kTriCols > kFusedMaxTiles) return 0;
  if (G > kTriRegG) return 0;  // the sweep holds every band's sums in registers
  const int cmax = G < kFusedMaxCluster ? G : kFusedMaxCluster;
  int cl = 0;
  for (int c = 1; c <= cmax && !cl; ++c)
    if (L::bytes(P->W, (G + c - 1) / c, srows, P->M) <= kFusedSmemTwoPerSM) cl = c;
  if (!cl && L::bytes(P->W, (G + cmax - 1) / cmax, srows, P->M) <= kFusedSmemMax) cl = cmax;
  if (!cl) return 0;
  if ((long)nf * cl < 2L * sms) cl = cmax;
  *gc_out = (G + cl - 1) / cl;
  *smem_out = L::bytes(P->W, *gc_out, srows, P->M);
  // Each CTA runs its bands one after another with the field's spectrum held
  // in shared memory (two CTAs per SM at most). Measured against the three
  // persistent launches, the fused solve wins only where every CTA holds a
  // single band (at most 8 bands: 72 x 108, 16.5 against 24 us for one field)
  // and the launch is latency-bound (its CTAs take at most 7/8 of the GPU's
  // slots); with 2 to 4 bands per CTA it loses (270 x 270: 41 against 32 us).
  // GFC_FUSED_SMALL=1 takes the fused solve wherever it applies.
  const int per_sm = *smem_out <= kFusedSmemTwoPerSM ? 2 : 1;
  if ((*gc_out > 1 || (long)nf * cl * 8 > (long)per_sm * sms * 7) && getenv("GFC_FUSED_SMALL") == nullptr) return 0;
  return cl;
}

// The fused solve from gradients on `nf` fields of a recursive-column-solve
// plan; cudaErrorNotSupported where it does not apply (the caller runs the
// three-step path) or when GFC_UNFUSED_SMALL is set.
template <class RS, typename T>
static cudaError_t run_fused_small(gfc_plan* P, const T* gx, const T* gy, T* out, int nf, cudaStream_t st) {
  if (!P->tri || P->pad != kP || getenv("GFC_UNFUSED_SMALL") != nullptr) return cudaErrorNotSupported;
  // by default only tori of at most 8 bands qualify (one band per CTA, see
  // fused_small_cluster): most plans stop here, before any runtime call
  if (P->triG > kFusedMaxCluster && getenv("GFC_FUSED_SMALL") == nullptr) return cudaErrorNotSupported;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int sms_of[64] = {};  // SM count per device, read once (relaxed atomics: every writer stores the same value)
  int sms = dev < 64 ? __atomic_load_n(&sms_of[dev], __ATOMIC_RELAXED) : 0;
  if (sms == 0) {
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (dev < 64) __atomic_store_n(&sms_of[dev], sms, __ATOMIC_RELAXED);
  }
  int gc = 0;
  size_t smem = 0;
  const int cl = fused_small_cluster<RS, T>(P, nf, sms, &gc, &smem);
  if (cl == 0) return cudaErrorNotSupported;
  FastArgs A;
  A.stage_out = 0;
  A.invM = 1.0 / (double)P->M;
  A.invN = 1.0 / (double)P->N;
  A.adj = 0;
  A.l2res = 0;
  A.H = P->H; A.W = P->W; A.p = P->pad; A.M = P->M; A.N = P->N; A.Nh = P->Nh; A.ldM = P->ldM;
  A.nrows = P->H + 1;
  A.ncols = P->W + 1;
  A.npairs = (A.nrows + 1) / 2;
  A.ldz = (RS::N + 3) & ~3;
  A.ngroups = P->triG;
  A.zpairs = A.ngroups * RS::F;
  A.nparts = 0;
  A.nf = nf;
  A.ldY = RS::LDY;
  A.err = P->dev_err;
  A.srows = 2 * A.zpairs;
  A.G = P->triG;
  A.tri_field = 0;
  if (A.ldY != ((P->Nh + 3) & ~3)) return cudaErrorNotSupported;
  auto kern = k_fused_small<RS, T>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(nf * cl));
  cfg.blockDim = dim3(RS::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  {
    // per (device, cluster size, shared memory): can such clusters be resident at all
    // (the kernel's dynamic shared-memory cap is raised to the largest size
    // launched so far on the device; the cap plus the static part must stay
    // within the per-block opt-in limit)
    static std::mutex mu;
    static std::map<std::pair<int, std::pair<int, size_t>>, int> fits;
    static std::map<int, size_t> cap;
    std::lock_guard<std::mutex> lock(mu);
    if (cap[dev] < smem) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        (void)cudaGetLastError();
        return cudaErrorNotSupported;
      }
      cap[dev] = smem;
    }
    const auto key = std::make_pair(dev, std::make_pair(cl, smem));
    auto it = fits.find(key);
    if (it == fits.end()) {
      int n = 0;
      if ((e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg)) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
      }
      it = fits.emplace(key, n).first;
    }
    if (it->second < 1) return cudaErrorNotSupported;
  }
  prof_begin(P, 0, st);
  e = cudaLaunchKernelEx(&cfg, kern, gx, gy, out, static_cast<const float2*>(P->twN),
                         static_cast<const float*>(P->colcoef), A, cl, gc);
  prof_end(P, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace gfc

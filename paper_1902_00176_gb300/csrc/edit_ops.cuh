// edit_ops.cuh -- per-pixel gradient edits (Sec. 3.2.3 thresholding, Eq. 26
// merging), shared by the standalone editing kernels and the divergence passes
// that apply an edit as they load the gradient. Every operation is written with
// explicitly rounded intrinsics, so both places compute the same bits whatever
// the compiler contracts elsewhere.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace gfc {

enum EditKind { kEditNone = 0, kEditThreshold = 1, kEditMerge = 2 };

// The edit of one solve call, as the divergence pass sees it.
struct EditArgs {
  int kind;           // EditKind
  float alpha;        // merge weight (Eq. 26)
  const void* edges;  // merge: edge map at the chunk's first field (plan dtype)
  const float* t2;    // threshold: squared threshold of each field of the chunk
  // colour correction (Eq. 25) fused after the solve: the statistics of the
  // solved field are taken as pass C stores it; null = none
  const float* ref_mean;  // reference mean of each field of the chunk
  const float* ref_std;   // reference standard deviation of each field of the chunk
};

// |E|^2 with both products and the sum rounded to FP32 (no contraction)
__device__ __forceinline__ float edit_mag2(float x, float y) { return __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)); }

// Eq. 26 as a factor on E: (C / |E|)^alpha = exp2(alpha (log2 C - log2(|E|^2) / 2));
// 0 where |E| = 0 (no orientation) or C = 0 (alpha > 0); 1 for alpha = 0.
__device__ __forceinline__ float edit_merge_scale(float x, float y, float c, float alpha) {
  const float m2 = edit_mag2(x, y);
  if (m2 == 0.0f) return 0.0f;
  if (alpha == 0.0f) return 1.0f;
  if (!(c > 0.0f)) return 0.0f;
  return exp2f(__fmul_rn(alpha, __fsub_rn(log2f(c), __fmul_rn(0.5f, log2f(m2)))));
}

__device__ __forceinline__ float edit_ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float edit_ld(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float edit_ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// the value a store to T followed by a load gives back
__device__ __forceinline__ float edit_round(float x, const float*) { return x; }
__device__ __forceinline__ float edit_round(float x, const __half*) { return __half2float(__float2half_rn(x)); }
__device__ __forceinline__ float edit_round(float x, const __nv_bfloat16*) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// Edited gradient (Ex, Ey) at pixel (i, j) of an H x W field; 0 outside the field.
// Equal, bit for bit, to what the standalone edit stores and a later pass loads.
template <typename T, int EDIT>
__device__ __forceinline__ float2 edit_pixel(const T* __restrict__ gx, const T* __restrict__ gy,
                                             const T* __restrict__ edges, int i, int j, int H, int W, float t2,
                                             float alpha) {
  if (i < 0 || i >= H || j < 0 || j >= W) return make_float2(0.0f, 0.0f);
  const size_t o = (size_t)i * W + j;
  const float x = edit_ld(gx + o), y = edit_ld(gy + o);
  if (EDIT == kEditThreshold) {
    const bool drop = edit_mag2(x, y) < t2;
    return drop ? make_float2(0.0f, 0.0f) : make_float2(x, y);
  } else if (EDIT == kEditMerge) {
    const float s = edit_merge_scale(x, y, edit_ld(edges + o), alpha);
    return make_float2(edit_round(__fmul_rn(x, s), gx), edit_round(__fmul_rn(y, s), gx));
  } else {
    return make_float2(x, y);
  }
}

}  // namespace gfc

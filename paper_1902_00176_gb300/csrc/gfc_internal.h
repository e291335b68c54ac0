// gfc_internal.h -- plan object and host helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gfc.h"
#include "edit_ops.cuh"
#include "fft_core.cuh"

namespace gfc {
// Row lengths with register-resident row passes, ascending: the SMOOTH size
// policy picks N from them (the smallest >= W + 2p when W + 2p lies in
// (kRowPolicyMin, last]), and the row kernels take the narrowest image that
// maps to their N from them. solve_fast.cu registers a kernel set for each.
constexpr int kRowLengthList[] = {108,  140,  160,  180,  200,  224,  252,  270,  294,  320,  360,
                                  400,  448,  500,  560,  630,  700,  784,  882,  980,  1080, 1120,
                                  1200, 1250, 1372, 1400, 1536, 1568, 1750, 1960, 2058};
constexpr int kRowPolicyMin = 136;

constexpr bool cx_is_smooth7(int n) {
  if (n < 1) return false;
  for (int f : {2, 3, 5, 7})
    while (n % f == 0) n /= f;
  return n == 1;
}
constexpr int cx_smooth_even_at_least(int x) {
  int n = x + (x & 1);
  while (!cx_is_smooth7(n)) n += 2;
  return n;
}
// the SMOOTH policy's row length for W + 2p = n
constexpr int cx_row_policy(int n) {
  constexpr int last = kRowLengthList[sizeof(kRowLengthList) / sizeof(int) - 1];
  if (n > kRowPolicyMin && n <= last)
    for (int r : kRowLengthList)
      if (r >= n) return r;
  return cx_smooth_even_at_least(n);
}

// scratch of one chunk in flight
struct Bufs {
  float2* spec;    // spectrum
  float2* zbuf;    // packed rows of L / row-major spectrum (fast passes)
  float* partial;  // per-block sums
  float2* tri;     // band sums and carries of the recursive column solve (fast passes)
};
constexpr int kMaxSlots = 4;
// L2 the spectrum hand-off of the chunks in flight may take (of the GPU's
// 126 MB): below it, the row pass writes the spectrum with an evict-last
// policy, gradients stream with evict-first and the inverse row pass drops the
// spectrum lines it has read, so the hand-off need not reach HBM
constexpr size_t kL2ResidentBytes = (size_t)80 << 20;
constexpr int kMaxRagStreams = 8;  // streams of a ragged plan's per-item sub-plans
constexpr int kHostBufs = 4;  // most staging buffers of the host-buffer pipeline

// One transform length of an EXACT-size plan (exact.cu).
struct ExactDim {
  int n;          // transform length
  int L;          // Bluestein convolution length (7-smooth, >= 2n - 1); 0 when n itself is 7-smooth
  FftPlan plan;   // schedule of n (direct) or of L (Bluestein)
  float2* tw;     // roots of unity of the scheduled length
  float2* chirp;  // [n] exp(-i pi j^2 / n)            (Bluestein only)
  float2* cf;     // [L] DFT of the conjugate chirp / L (Bluestein only)
};

// One field (item, channel) of a ragged batch, as the generic passes read it.
struct FieldDesc {
  long long in_off;    // element offset of the field in the caller's arrays
  long long spec_off;  // complex offset of its spectrum in the chunk scratch
  long long G_off;     // float offset of its Green table in the pool
  int H, W, M, N, Nh, ldS;
  int twN_off, twM_off;  // float2 offsets of its twiddle tables in the pool
  int plan;              // index of its (row, column) transform schedules
  int pad;
};
}  // namespace gfc

struct gfc_plan {
  // problem
  int H, W, C, batch, pad;
  gfc_dtype dtype;
  int M, N;   // padded (torus) size
  int Nh;     // N/2 + 1 Hermitian columns
  int ldS;    // row stride of the row-major spectrum scratch (generic passes), complex elements
  int ldM;    // column stride of the column-major spectrum scratch (fast passes)
  bool fast;  // the row length has register-resident passes (fast_kernels.cuh)
  bool fast_cols;  // ... and the column length has them too (column FFT path, adjoint)
  bool tri;   // fast passes with the column direction by recursive filters (gfc_column_solver)
  bool block_items;  // fast passes launch one block per item (else persistent grids)
  bool l2res;        // recursive column solve whose spectrum hand-off (chunk x streams) fits kL2ResidentBytes
  int triG;   // bands of the recursive column solve (pass A's items)
  size_t tri_field;  // complex elements per field of the band scratch
  float* colcoef;    // [Nh][8] column coefficients of the recursive solve
  float* powc;       // [2 triG][ldS] carry weights of the bands
  int triGh;         // half-bands of F rows (the adjoint's recursive column solve)
  float* colcoef_h;  // colcoef and powc for the half-bands
  float* powc_h;
  float2* tri_buf;   // [slots][chunk][tri_field] band scratch
  bool exact; // size policy EXACT: M = H + 2p, N = W + 2p (exact.cu)
  gfc::ExactDim ex_row, ex_col;  // EXACT: the length-N and length-M transforms
  int chunk;  // fields per pipeline chunk
  int device;
  cudaStream_t stream;
  // FFT schedules
  gfc::FftPlan rowplan;  // length N
  gfc::FftPlan colplan;  // length M
  // device tables (owned)
  float* G;       // [M][Nh] Green spectrum with 1/(MN) folded in
  float* GT;      // [Nh][ldM] the same, transposed (fast passes)
  float2* twN;    // [N] exp(-2 pi i m / N)
  float2* twM;    // [M] exp(-2 pi i m / M)
  float2* spec;   // [slots][chunk] spectrum scratch (per field: max(M ldS, Nh ldM) complex)
  float* partial; // [slots][chunk][kMaxRowBlocks] per-block sums (adjoint, u[0,0])
  float* edit_t2; // [batch * C] squared gradient threshold per field (Sec. 3.2.3)
  float2* zbuf;   // [slots][chunk] packed rows of L / row-major spectrum (fast passes)
  size_t spec_field, zbuf_field;  // elements per field of spec and zbuf
  int nslots;                     // chunks in flight
  cudaStream_t slot_stream[gfc::kMaxSlots];
  cudaEvent_t slot_done[gfc::kMaxSlots];
  cudaEvent_t ev_fork;
  int* dev_err;   // device error word
  // host-buffer path (allocated on first use)
  void* stage_in[gfc::kHostBufs][2];  // [buffer][gx, gy] device staging for one host step
  void* stage_out[gfc::kHostBufs];
  cudaStream_t copy_in, copy_out;
  cudaEvent_t ev_in[gfc::kHostBufs], ev_comp[gfc::kHostBufs], ev_out[gfc::kHostBufs];
  int host_bufs;          // staging buffers in rotation (<= kHostBufs)
  bool host_ready;
  int host_chunk;         // fields per host-pipeline step (copies of one step overlap the solve of another)
  // ragged batch (gfc_plan_create_ragged)
  bool ragged;
  int nfields;               // total fields (sum of item channels)
  int nchunks;               // chunks of fields processed one after another
  int* chunk_begin;          // [nchunks + 1] host: first field of each chunk
  gfc::FieldDesc* d_desc;    // [nfields] device
  gfc::FftPlan* d_plans;     // [2 * sizes] device: row, column schedule per distinct size
  int maxM, maxN, maxNh, maxH, maxW;
  // ragged batches on the register-resident passes: one uniform sub-plan per item
  // (batch 1, the item's C), run on rag_streams internal streams forked from and
  // joined into the plan's stream; the other items (nfields of them) go through
  // the generic per-field passes above
  int nsub;
  gfc_plan** sub;          // [nsub]
  long long* sub_off;      // [nsub] element offset of each sub-plan's item in the packed arrays
  int* sub_stream;         // [nsub] the stream each sub-plan runs on
  double* sub_work;        // [nsub] the item's size (C H W), for the stream assignment
  long long rag_total;      // elements of the packed arrays the items span
  int rag_streams;          // streams created
  int rag_active;           // streams the sub-plans are spread over (<= rag_streams)
  cudaStream_t rag_stream[gfc::kMaxRagStreams];
  cudaEvent_t rag_done[gfc::kMaxRagStreams];
  cudaEvent_t rag_fork;
  // tracing
  gfc_profile prof;
  bool profiling;
  int ev_cap, ev_used;
  cudaEvent_t* ev_start;
  cudaEvent_t* ev_stop;
  int* ev_pass;
};

namespace gfc {

constexpr int kMaxRowBlocks = 2048;

// thread-local error text, set by fail()
gfc_status fail(gfc_status s, const char* fmt, ...);
gfc_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

// mixed-radix schedule for a 7-smooth n (returns false if n is not 7-smooth or too long)
bool make_fft_plan(int n, FftPlan* pl);
bool is_7smooth(long n);

// device table builders (FP64 on the GPU, rounded to FP32)
cudaError_t build_twiddles(float2* tw, int n, cudaStream_t s);
cudaError_t build_green(float* G, int M, int N, int Nh, cudaStream_t s);
cudaError_t build_green_t(float* GT, int M, int N, int Nh, int ldM, cudaStream_t s);
// recursive column solve tables: cc [Nh][8], pw [tri_power_rows(G)][ldY] (bands of `band` rows
// from row `pad`; the carry sweep cuts the G bands into 8 segments)
constexpr int kTriSegments = 8;
inline int tri_power_rows(int G) { return (G + kTriSegments - 1) / kTriSegments + 1; }
cudaError_t build_colcoef(float* cc, float* pw, int M, int N, int Nh, int ldY, int pad, int G, int band,
                          cudaStream_t s);

// register-resident passes (solve_fast.cu): spectrum laid out [l][r]
bool fast_supported(int M, int N);      // row and column passes compiled for M x N
bool fast_rows_supported(int N);        // row passes compiled for N alone (recursive column solve, FP32)
int fast_row_lengths(int* out, int cap);  // compiled row lengths, ascending; returns the count
size_t fast_zbuf_elems(int H, int M, int N);  // per field
int fast_row_items(int M, int N);             // row pairs per item of the row passes (F)
// mode 0 gradient, 1 Laplacian, 2 adjoint (out1 = grad_gy)
// `ed` (mode 0 only, may be null) applies a gradient edit as the gradient is loaded
cudaError_t run_chunk_fast(gfc_plan* P, const Bufs& B, int mode, const void* in0, const void* in1, void* out0,
                           void* out1, int nf, cudaStream_t st, const EditArgs* ed = nullptr);
inline Bufs slot_bufs(const gfc_plan* P, int s) {
  Bufs b;
  b.spec = P->spec + (size_t)s * P->chunk * P->spec_field;
  b.zbuf = P->zbuf ? P->zbuf + (size_t)s * P->chunk * P->zbuf_field : nullptr;
  b.partial = P->partial + (size_t)s * P->chunk * kMaxRowBlocks;
  b.tri = P->tri_buf ? P->tri_buf + (size_t)s * P->chunk * P->tri_field : nullptr;
  return b;
}

inline size_t dtype_size(gfc_dtype d) { return d == GFC_F32 ? 4 : 2; }

// tracing around one kernel launch on the plan's stream
void prof_begin(gfc_plan* P, int pass, cudaStream_t st);
void prof_end(gfc_plan* P, cudaStream_t st);
// EXACT-size plans (exact.cu): tables, teardown, one chunk (mode 0 gradient,
// 1 Laplacian, 2 adjoint into out0 = grad_gx, out1 = grad_gy; `ed` as for
// run_chunk_fast). The chunk scratch holds 2 M N complex per field.
cudaError_t exact_setup(gfc_plan* P, cudaStream_t s);
void exact_release(gfc_plan* P);
cudaError_t run_chunk_exact(gfc_plan* P, const Bufs& B, int mode, const void* in0, const void* in1, void* out0,
                            void* out1, int nf, cudaStream_t st, const EditArgs* ed);

// per-field squared thresholds of Sec. 3.2.3 into P->edit_t2 (edit.cu): from
// the fields' largest gradient magnitudes when ref <= 0, else from ref
gfc_status edit_prepare_threshold(gfc_plan* P, const void* gx, const void* gy, float frac, float ref);

// spread a ragged plan's sub-plans over k internal streams (plan.cu)
gfc_status ragged_set_streams(gfc_plan* P, int k);

// free the host-buffer pipeline and the profiling event pool (plan teardown)
void release_host_state(gfc_plan* P);

// spectrum hand-off bytes per field of a solve on a recursive-column-solve
// plan: the row-major spectrum S (2F rows per band), the bands' carries and
// sums, column 0's compact copy
inline size_t tri_handoff_bytes(const gfc_plan* p) {
  const size_t G = (size_t)p->triG, srows = (size_t)2 * fast_row_items(p->M, p->N) * G;
  const size_t nkb = ((size_t)p->ldS + 31) / 32;
  return (srows * p->ldS + 2 * G * p->ldS + nkb * 2 * G * 32) * sizeof(float2) + srows * sizeof(float);
}

}  // namespace gfc

#define GFC_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return gfc::cuda_fail(e_, #expr); \
  } while (0)

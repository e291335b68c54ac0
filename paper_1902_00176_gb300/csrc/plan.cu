// plan.cu -- plan creation, size policy, FP64 table builders, status/error plumbing.
//
// Algorithm A of the paper builds the Green spectrum once per image size as
// fft(dirac)/fft(laplace) with both kernels centred at [1,1]. The phases
// cancel, so the spectrum is real: G[k,l] = 1/lambda(k,l) with
// lambda = 2cos(2 pi k/M) + 2cos(2 pi l/N) - 4 = -4 (sin^2(pi k/M) + sin^2(pi l/N)).
// The plan evaluates the sin^2 form in FP64 on the GPU (no cancellation near
// DC), folds in the inverse transform's 1/(MN), stores FP32, and sets the DC
// bin (0/0 in Algorithm A) to 0.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "gfc_internal.h"

namespace gfc {

static thread_local char g_err[512] = "";

void clear_error() { g_err[0] = '\0'; }

gfc_status fail(gfc_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

gfc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? GFC_ERR_ALLOC : GFC_ERR_CUDA, "%s: %s (%s)", what,
              cudaGetErrorString(e), cudaGetErrorName(e));
}

bool is_7smooth(long n) {
  if (n < 1) return false;
  for (long f : {2L, 3L, 5L, 7L})
    while (n % f == 0) n /= f;
  return n == 1;
}

// Stage order: the power of two as radix-8 stages plus one radix-4 or radix-2
// stage, then 3s, 5s and 7s. Any order is a valid Stockham schedule.
bool make_fft_plan(int n, FftPlan* pl) {
  if (n < 1 || n > kMaxFftLen || !is_7smooth(n)) return false;
  int m = n, e2 = 0;
  while (m % 2 == 0) { m /= 2; ++e2; }
  int ns = 0;
  while (e2 >= 3) { pl->radix[ns++] = 8; e2 -= 3; }
  if (e2 == 2) pl->radix[ns++] = 4;
  if (e2 == 1) pl->radix[ns++] = 2;
  for (int f : {3, 5, 7})
    while (m % f == 0) {
      if (ns >= kMaxStages) return false;
      pl->radix[ns++] = f;
      m /= f;
    }
  pl->n = n;
  pl->nst = ns;
  return true;
}

__global__ void k_build_twiddles(float2* tw, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)(-s));
  }
}

__global__ void k_build_green(float* G, int M, int N, int Nh) {
  const long total = (long)M * Nh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / Nh), l = (int)(idx % Nh);
    const double sk = sinpi((double)k / (double)M), sl = sinpi((double)l / (double)N);
    const double lam = -4.0 * (sk * sk + sl * sl);
    G[idx] = (k == 0 && l == 0) ? 0.0f : (float)(1.0 / (lam * (double)M * (double)N));
  }
}

__global__ void k_build_green_t(float* GT, int M, int N, int Nh, int ldM) {
  const long total = (long)Nh * ldM;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int l = (int)(idx / ldM), k = (int)(idx % ldM);
    if (k >= M) {
      GT[idx] = 0.0f;
      continue;
    }
    const double sk = sinpi((double)k / (double)M), sl = sinpi((double)l / (double)N);
    const double lam = -4.0 * (sk * sk + sl * sl);
    GT[idx] = (k == 0 && l == 0) ? 0.0f : (float)(1.0 / (lam * (double)M * (double)N));
  }
}

// Coefficients of the recursive column solve, per Hermitian column l (FP64,
// rounded once to FP32). After the row transforms, column l of Eq. 23's
// Green multiply is the inverse of the cyclic tridiagonal operator
// S + S^-1 - b_l along the torus rows (S the row shift, b_l = 4 - 2 cos(2 pi l / N),
// i.e. lambda(k, l) = 2 cos(2 pi k / M) - b_l). With a_l + 1/a_l = b_l, a_l < 1,
//   (S + S^-1 - b)^-1 = -a / (1 - a^2) [ (1 - a S)^-1 + (1 - a S^-1)^-1 - 1 ],
// two first-order recursions (causal and anticausal) on the cyclic rows. The
// rows are cut into bands of `band` rows from torus row `pad` (the last one
// `last` rows long), followed by `tail` zero rows and the `pad` zero rows that
// close the cycle. Row l of the table: delta = 1 - a (formed without
// cancellation, so the pole stays exact near DC), a, C = -a / ((1 - a^2) N)
// (1/N: the unnormalised inverse row transform), a^band, a^last, a^pad,
// 1 / (1 - a^M), a^tail. Column 0 (b = 2, singular) is solved exactly
// elsewhere; its row is zero.
// After the [Nh][8] rows, `dc` holds (delta, C) of every column compactly,
// [ldY][2] (zero past Nh), for the in-band recursions of the inverse row pass.
__global__ void k_build_colcoef(float* cc, float* dc, int M, int N, int Nh, int ldY, int pad, int band, int last,
                                int tail) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ldY; l += gridDim.x * blockDim.x) {
    if (l >= Nh || l == 0) {
      dc[2 * l] = dc[2 * l + 1] = 0.0f;
      if (l == 0)
        for (int i = 0; i < 8; ++i) cc[i] = 0.0f;
      continue;
    }
    float* c = cc + (size_t)l * 8;
    const double sn = sinpi((double)l / (double)N);
    const double d = 4.0 * sn * sn;  // b - 2
    const double r = sqrt(d * (4.0 + d));
    const double a = 2.0 / (2.0 + d + r), delta = (d + r) / (2.0 + d + r);
    c[0] = (float)delta;
    c[1] = (float)a;
    c[2] = (float)(-a / (delta * (1.0 + a) * (double)N));
    c[3] = (float)pow(a, (double)band);
    c[4] = (float)pow(a, (double)last);
    c[5] = (float)pow(a, (double)pad);
    c[6] = (float)(1.0 / (1.0 - pow(a, (double)M)));
    c[7] = (float)pow(a, (double)tail);
    dc[2 * l] = c[0];
    dc[2 * l + 1] = c[2];
  }
}

// Segment transfers of the carry sweep, [rows][ldY]: row r holds a^(band r),
// the transfer of r full bands (FP64, rounded once).
__global__ void k_build_powc(float* pw, int N, int Nh, int ldY, int rows, int band) {
  const long total = (long)rows * ldY;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ldY), l = (int)(idx % ldY);
    if (l == 0 || l >= Nh) {
      pw[idx] = 0.0f;
      continue;
    }
    const double sn = sinpi((double)l / (double)N);
    const double d = 4.0 * sn * sn;
    const double a = 2.0 / (2.0 + d + sqrt(d * (4.0 + d)));
    pw[idx] = (float)pow(a, (double)band * r);
  }
}

cudaError_t build_colcoef(float* cc, float* pw, int M, int N, int Nh, int ldY, int pad, int G, int band,
                          cudaStream_t s) {
  const int last = (M - pad - band * (G - 1)) < band ? (M - pad - band * (G - 1)) : band;
  const int tail = (M - pad - band * G) > 0 ? (M - pad - band * G) : 0;
  k_build_colcoef<<<(ldY + 255) / 256, 256, 0, s>>>(cc, cc + (size_t)Nh * 8, M, N, Nh, ldY, pad, band, last, tail);
  const int rows = tri_power_rows(G);
  const long total = (long)rows * ldY;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_build_powc<<<blocks, 256, 0, s>>>(pw, N, Nh, ldY, rows, band);
  return cudaGetLastError();
}

cudaError_t build_green_t(float* GT, int M, int N, int Nh, int ldM, cudaStream_t s) {
  long total = (long)Nh * ldM;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_build_green_t<<<blocks, 256, 0, s>>>(GT, M, N, Nh, ldM);
  return cudaGetLastError();
}

cudaError_t build_twiddles(float2* tw, int n, cudaStream_t s) {
  k_build_twiddles<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
  return cudaGetLastError();
}

cudaError_t build_green(float* G, int M, int N, int Nh, cudaStream_t s) {
  long total = (long)M * Nh;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_build_green<<<blocks, 256, 0, s>>>(G, M, N, Nh);
  return cudaGetLastError();
}

static int smooth_even_at_least(int x) {
  int n = x + (x & 1);
  while (!is_7smooth(n)) n += 2;
  return n;
}

}  // namespace gfc

using namespace gfc;

static void destroy_plan(gfc_plan* p);

extern "C" {

const char* gfc_last_error(void) { return g_err; }

const char* gfc_status_string(gfc_status s) {
  switch (s) {
    case GFC_OK: return "GFC_OK";
    case GFC_ERR_INVALID_ARG: return "GFC_ERR_INVALID_ARG";
    case GFC_ERR_UNSUPPORTED: return "GFC_ERR_UNSUPPORTED";
    case GFC_ERR_ALLOC: return "GFC_ERR_ALLOC";
    case GFC_ERR_CUDA: return "GFC_ERR_CUDA";
    case GFC_ERR_TIMEOUT: return "GFC_ERR_TIMEOUT";
  }
  return "GFC_ERR_UNKNOWN";
}

gfc_status gfc_padded_size(int H, int W, int pad, int size_policy, int* M, int* N) {
  clear_error();
  if (!M || !N) return fail(GFC_ERR_INVALID_ARG, "gfc_padded_size: null output pointer");
  if (H < 2 || W < 2) return fail(GFC_ERR_INVALID_ARG, "gfc_padded_size: H=%d W=%d (need >= 2)", H, W);
  if (pad <= 0) pad = 4;
  if (size_policy == GFC_SIZE_EXACT) {
    // Algorithm A's size; Bluestein's convolution length stays <= kMaxFftLen
    if ((long)H + 2L * pad > kMaxFftLen / 2 || (long)W + 2L * pad > kMaxFftLen / 2)
      return fail(GFC_ERR_UNSUPPORTED, "gfc_padded_size: exact size %ldx%ld exceeds %d", (long)H + 2L * pad,
                  (long)W + 2L * pad, kMaxFftLen / 2);
    *M = H + 2 * pad;
    *N = W + 2 * pad;
    return GFC_OK;
  }
  if (size_policy != GFC_SIZE_SMOOTH)
    return fail(GFC_ERR_INVALID_ARG, "gfc_padded_size: unknown size policy %d", size_policy);
  if ((long)H + 2L * pad > kMaxFftLen || (long)W + 2L * pad > kMaxFftLen)
    return fail(GFC_ERR_UNSUPPORTED, "gfc_padded_size: H+2p=%ld or W+2p=%ld exceeds %d", (long)H + 2L * pad,
                (long)W + 2L * pad, kMaxFftLen);
  // M: the smallest even 7-smooth length; N: the smallest row length with
  // register-resident passes when W + 2p lies in their range, else as M
  const int m = smooth_even_at_least(H + 2 * pad), n = cx_row_policy(W + 2 * pad);
  if (m > kMaxFftLen || n > kMaxFftLen)
    return fail(GFC_ERR_UNSUPPORTED, "gfc_padded_size: padded size %dx%d exceeds %d", m, n, kMaxFftLen);
  *M = m;
  *N = n;
  return GFC_OK;
}

int gfc_plan_l2_resident(const gfc_plan* plan) {
  clear_error();
  return plan ? (plan->l2res ? 1 : 0) : -1;
}

int gfc_row_lengths(int* lengths, int capacity) {
  clear_error();
  return fast_row_lengths(lengths, lengths ? capacity : 0);
}

gfc_status gfc_plan_create_ex(gfc_plan** out, const gfc_plan_opts* o) {
  clear_error();
  if (!out || !o) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create: null argument");
  *out = nullptr;
  if (o->C < 1 || o->batch < 1)
    return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create: C=%d batch=%d (need >= 1)", o->C, o->batch);
  if (o->dtype != GFC_F32 && o->dtype != GFC_F16 && o->dtype != GFC_BF16)
    return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create: unknown dtype %d", (int)o->dtype);
  if (o->chunk < 0) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create: chunk=%d", o->chunk);
  int M, N;
  gfc_status st = gfc_padded_size(o->H, o->W, o->pad, o->size_policy, &M, &N);
  if (st != GFC_OK) return st;
  const int pad = o->pad <= 0 ? 4 : o->pad;

  gfc_plan* p = (gfc_plan*)calloc(1, sizeof(gfc_plan));
  if (!p) return fail(GFC_ERR_ALLOC, "gfc_plan_create: host allocation failed");
  p->H = o->H; p->W = o->W; p->C = o->C; p->batch = o->batch; p->pad = pad; p->dtype = o->dtype;
  p->M = M; p->N = N; p->Nh = N / 2 + 1; p->ldS = (p->Nh + 3) & ~3; p->ldM = (M + 3) & ~3;
  p->exact = o->size_policy == GFC_SIZE_EXACT;
  if (o->column_solver != GFC_COLUMN_RECURSIVE && o->column_solver != GFC_COLUMN_FFT) {
    free(p);
    return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create: unknown column solver %d", o->column_solver);
  }
  const bool usable = !p->exact && pad == 4 && getenv("GFC_FORCE_GENERIC") == nullptr;
  p->fast_cols = usable && fast_supported(M, N);
  // row-only lengths run FP32 with the recursive column solve
  const bool rows_only = usable && !p->fast_cols && fast_rows_supported(N) && o->dtype == GFC_F32 &&
                         o->column_solver == GFC_COLUMN_RECURSIVE;
  p->fast = p->fast_cols || rows_only;
  p->tri = p->fast && o->column_solver == GFC_COLUMN_RECURSIVE;
  p->block_items = o->block_items != 0;
  if (p->tri) {
    const int F = fast_row_items(M, N);
    p->triG = (((o->H + 2) / 2) + F - 1) / F;
    // the adjoint sweeps half-bands of F rows (those that start on the torus)
    const int halves = (M - pad + F - 1) / F;
    p->triGh = 2 * p->triG < halves ? 2 * p->triG : halves;
    // carries [G][2][ldS], band sums in 32-column tiles, column 0 of the 2 F G rows
    // of S as floats (G: bands, or half-bands for the adjoint, whichever is more);
    // even, so every field's scratch stays 16-byte aligned
    const size_t nkb = (size_t)(p->ldS + 31) / 32;
    const size_t gmax = p->triGh > p->triG ? p->triGh : p->triG;
    p->tri_field = ((size_t)2 * gmax * p->ldS + nkb * 2 * gmax * 32 + (size_t)(2 * F * p->triG + 1) / 2 + 1) &
                   ~(size_t)1;
  }
  p->stream = (cudaStream_t)o->stream;
  if (!p->exact && (!make_fft_plan(N, &p->rowplan) || !make_fft_plan(M, &p->colplan))) {
    free(p);
    return fail(GFC_ERR_UNSUPPORTED, "gfc_plan_create: no FFT schedule for %dx%d", M, N);
  }
  if (o->streams < 0 || o->streams > kMaxSlots) {
    free(p);
    return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create: streams=%d (0..%d)", o->streams, kMaxSlots);
  }
  const long fields = (long)o->batch * o->C;
  const size_t per_row_major = (size_t)M * p->ldS, per_col_major = (size_t)p->Nh * p->ldM;
  p->spec_field = per_row_major > per_col_major ? per_row_major : per_col_major;
  if (p->exact) p->spec_field = 2 * (size_t)M * N;  // the complex torus and its transpose
  p->zbuf_field = p->fast ? fast_zbuf_elems(o->H, M, N) : 0;
  if (p->tri) {  // the row-major spectrum holds 2F rows per band
    const size_t srows = (size_t)2 * fast_row_items(M, N) * p->triG * p->ldS;
    if (srows > p->spec_field) p->spec_field = srows;
  }
  const size_t per_field = p->spec_field * sizeof(float2);
  const size_t ws = per_field + (p->zbuf_field + p->tri_field) * sizeof(float2);
  long chunk = o->chunk;
  int nslots = o->streams;
  if (nslots == 0) nslots = 1;
  if (chunk == 0) {
    // Measured on GB300 (801x1200 fields): the passes are bound by arithmetic
    // and latency rather than by where the intermediates live, and large
    // grids beat L2-sized chunks (1.11 ms per 100 fields in one chunk, 1.29 -
    // 1.41 ms with 2 - 12 field chunks on 2 - 4 streams). So one chunk holds as
    // many fields as 2 GB of scratch allows.
    chunk = (long)((size_t(2) << 30) / (ws * nslots));
    if (chunk < 1) chunk = 1;
  }
  if (chunk > fields) chunk = fields;
  if (p->exact && chunk > 65535) chunk = 65535;  // fields are a grid dimension there
  const long nchunks = (fields + chunk - 1) / chunk;
  if (nslots > nchunks) nslots = (int)nchunks;
  p->chunk = (int)chunk;
  p->nslots = nslots;
  // the chunks in flight hand their spectra to the inverse row pass through L2
  p->l2res = p->tri && (size_t)chunk * nslots * tri_handoff_bytes(p) <= kL2ResidentBytes &&
             getenv("GFC_NO_L2RES") == nullptr;

  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->G, (size_t)M * p->Nh * sizeof(float));
  if (e == cudaSuccess && p->fast_cols) e = cudaMalloc(&p->GT, (size_t)p->Nh * p->ldM * sizeof(float));
  if (e == cudaSuccess && p->fast) e = cudaMalloc(&p->zbuf, p->zbuf_field * chunk * nslots * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->twN, (size_t)N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->twM, (size_t)M * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->spec, per_field * (size_t)chunk * nslots);
  if (e == cudaSuccess) e = cudaMalloc(&p->partial, (size_t)chunk * nslots * kMaxRowBlocks * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&p->edit_t2, (size_t)fields * sizeof(float));
  if (e == cudaSuccess && p->tri) e = cudaMalloc(&p->colcoef, ((size_t)p->Nh * 8 + 2 * (size_t)p->ldS) * sizeof(float));
  if (e == cudaSuccess && p->tri) e = cudaMalloc(&p->powc, (size_t)tri_power_rows(p->triG) * p->ldS * sizeof(float));
  if (e == cudaSuccess && p->tri)
    e = cudaMalloc(&p->colcoef_h, ((size_t)p->Nh * 8 + 2 * (size_t)p->ldS) * sizeof(float));
  if (e == cudaSuccess && p->tri) e = cudaMalloc(&p->powc_h, (size_t)tri_power_rows(p->triGh) * p->ldS * sizeof(float));
  // (+64 bytes: the sweep's bulk copy of a field's column 0 rounds up to 16 bytes)
  if (e == cudaSuccess && p->tri) e = cudaMalloc(&p->tri_buf, p->tri_field * chunk * nslots * sizeof(float2) + 64);
  for (int sl = 0; sl < nslots && e == cudaSuccess; ++sl) {
    e = cudaStreamCreateWithFlags(&p->slot_stream[sl], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->slot_done[sl], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&p->dev_err, sizeof(int));
  cudaStream_t bs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dev_err, 0, sizeof(int), bs);
  if (e == cudaSuccess) e = build_twiddles(p->twN, N, bs);
  if (e == cudaSuccess) e = build_twiddles(p->twM, M, bs);
  if (e == cudaSuccess) e = build_green(p->G, M, N, p->Nh, bs);
  if (e == cudaSuccess && p->fast_cols) e = build_green_t(p->GT, M, N, p->Nh, p->ldM, bs);
  if (e == cudaSuccess && p->tri)
    e = build_colcoef(p->colcoef, p->powc, M, N, p->Nh, p->ldS, pad, p->triG, 2 * fast_row_items(M, N), bs);
  if (e == cudaSuccess && p->tri)
    e = build_colcoef(p->colcoef_h, p->powc_h, M, N, p->Nh, p->ldS, pad, p->triGh, fast_row_items(M, N), bs);
  if (e == cudaSuccess && p->exact) e = exact_setup(p, bs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
  if (bs) cudaStreamDestroy(bs);
  if (e != cudaSuccess) {
    gfc_status s = cuda_fail(e, "gfc_plan_create");
    destroy_plan(p);
    return s;
  }
  *out = p;
  return GFC_OK;
}

}  // extern "C"

// The generic part of a ragged plan: per-field descriptors over the given items
// (n >= 1), pooled tables, chunked scratch.
static gfc_status create_ragged_generic(gfc_plan** out, int n, const gfc_item* items, gfc_dtype dtype) {
  *out = nullptr;
  if (dtype != GFC_F32 && dtype != GFC_F16 && dtype != GFC_BF16)
    return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create_ragged: unknown dtype %d", (int)dtype);
  const int pad = 4;
  // distinct padded sizes
  std::vector<std::pair<int, int>> sizes;
  std::vector<int> item_size(n);
  long long nfields = 0;
  for (int i = 0; i < n; ++i) {
    const gfc_item& it = items[i];
    if (it.C < 1 || it.offset < 0)
      return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create_ragged: item %d has C=%d offset=%lld", i, it.C, it.offset);
    int M, N;
    gfc_status st = gfc_padded_size(it.H, it.W, pad, GFC_SIZE_SMOOTH, &M, &N);
    if (st != GFC_OK) return st;
    int k = 0;
    while (k < (int)sizes.size() && sizes[k] != std::make_pair(M, N)) ++k;
    if (k == (int)sizes.size()) sizes.push_back({M, N});
    item_size[i] = k;
    nfields += it.C;
  }
  if (nfields > (1 << 24)) return fail(GFC_ERR_UNSUPPORTED, "gfc_plan_create_ragged: too many fields");
  // pooled tables and schedules
  std::vector<FftPlan> plans(2 * sizes.size());
  std::vector<int> twN_off(sizes.size()), twM_off(sizes.size());
  std::vector<long long> G_off(sizes.size());
  int tw_total = 0;
  long long g_total = 0;
  for (size_t k = 0; k < sizes.size(); ++k) {
    const int M = sizes[k].first, N = sizes[k].second;
    if (!make_fft_plan(N, &plans[2 * k]) || !make_fft_plan(M, &plans[2 * k + 1]))
      return fail(GFC_ERR_UNSUPPORTED, "gfc_plan_create_ragged: no FFT schedule for %dx%d", M, N);
    twN_off[k] = tw_total;
    tw_total += N;
    twM_off[k] = tw_total;
    tw_total += M;
    G_off[k] = g_total;
    g_total += (long long)M * (N / 2 + 1);
  }
  // field descriptors and chunks (spectrum scratch of a chunk <= 1 GB, <= 65535 fields)
  const long long budget = (1ll << 30) / (long long)sizeof(float2);
  std::vector<FieldDesc> desc((size_t)nfields);
  std::vector<int> chunk_begin(1, 0);
  long long used = 0, max_chunk = 0;
  int fidx = 0, maxM = 0, maxN = 0, maxH = 0, maxW = 0;
  for (int i = 0; i < n; ++i) {
    const gfc_item& it = items[i];
    const int k = item_size[i], M = sizes[k].first, N = sizes[k].second;
    const int Nh = N / 2 + 1, ldS = (Nh + 3) & ~3;
    const long long need = (long long)M * ldS;
    for (int c = 0; c < it.C; ++c, ++fidx) {
      const int in_chunk = fidx - chunk_begin.back();
      if (in_chunk > 0 && (used + need > budget || in_chunk >= 65535)) {
        chunk_begin.push_back(fidx);
        used = 0;
      }
      FieldDesc& d = desc[fidx];
      d.in_off = it.offset + (long long)c * it.H * it.W;
      d.spec_off = used;
      d.G_off = G_off[k];
      d.H = it.H; d.W = it.W; d.M = M; d.N = N; d.Nh = Nh; d.ldS = ldS;
      d.twN_off = twN_off[k]; d.twM_off = twM_off[k];
      d.plan = k;
      d.pad = pad;
      used += need;
      if (used > max_chunk) max_chunk = used;
    }
    if (M > maxM) maxM = M;
    if (N > maxN) maxN = N;
    if (it.H > maxH) maxH = it.H;
    if (it.W > maxW) maxW = it.W;
  }
  chunk_begin.push_back((int)nfields);
  int max_fields_chunk = 0;
  for (size_t c = 0; c + 1 < chunk_begin.size(); ++c)
    max_fields_chunk = std::max(max_fields_chunk, chunk_begin[c + 1] - chunk_begin[c]);

  gfc_plan* p = (gfc_plan*)calloc(1, sizeof(gfc_plan));
  if (!p) return fail(GFC_ERR_ALLOC, "gfc_plan_create_ragged: host allocation failed");
  p->ragged = true;
  p->H = maxH; p->W = maxW; p->C = 1; p->batch = (int)nfields; p->pad = pad; p->dtype = dtype;
  p->M = maxM; p->N = maxN; p->Nh = maxN / 2 + 1; p->ldS = (p->Nh + 3) & ~3; p->ldM = (maxM + 3) & ~3;
  p->maxM = maxM; p->maxN = maxN; p->maxNh = maxN / 2 + 1; p->maxH = maxH; p->maxW = maxW;
  p->nfields = (int)nfields;
  p->nchunks = (int)chunk_begin.size() - 1;
  p->chunk = max_fields_chunk;
  p->nslots = 1;
  p->spec_field = 0;
  p->chunk_begin = (int*)malloc(chunk_begin.size() * sizeof(int));
  if (!p->chunk_begin) {
    free(p);
    return fail(GFC_ERR_ALLOC, "gfc_plan_create_ragged: host allocation failed");
  }
  memcpy(p->chunk_begin, chunk_begin.data(), chunk_begin.size() * sizeof(int));
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->twN, (size_t)tw_total * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->G, (size_t)g_total * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_desc, desc.size() * sizeof(FieldDesc));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_plans, plans.size() * sizeof(FftPlan));
  if (e == cudaSuccess) e = cudaMalloc(&p->spec, (size_t)max_chunk * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->partial, (size_t)max_fields_chunk * kMaxRowBlocks * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&p->dev_err, sizeof(int));
  cudaStream_t bs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dev_err, 0, sizeof(int), bs);
  for (size_t k = 0; k < sizes.size() && e == cudaSuccess; ++k) {
    const int M = sizes[k].first, N = sizes[k].second;
    e = build_twiddles(p->twN + twN_off[k], N, bs);
    if (e == cudaSuccess) e = build_twiddles(p->twN + twM_off[k], M, bs);
    if (e == cudaSuccess) e = build_green(p->G + G_off[k], M, N, N / 2 + 1, bs);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_desc, desc.data(), desc.size() * sizeof(FieldDesc), cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_plans, plans.data(), plans.size() * sizeof(FftPlan), cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
  if (bs) cudaStreamDestroy(bs);
  if (e != cudaSuccess) {
    gfc_status st = cuda_fail(e, "gfc_plan_create_ragged");
    destroy_plan(p);
    return st;
  }
  *out = p;
  return GFC_OK;
}

// Ragged plans: FP32 items whose padded size has register-resident row passes
// run as uniform sub-plans (batch 1, the item's C) on internal streams; the
// others go through the generic per-field passes.
static gfc_status attach_subplans(gfc_plan* p, const std::vector<int>& fast_items, const gfc_item* items) {
  const int ns = (int)fast_items.size();
  p->nsub = 0;
  if (ns == 0) return GFC_OK;
  p->sub = (gfc_plan**)calloc((size_t)ns, sizeof(gfc_plan*));
  p->sub_off = (long long*)calloc((size_t)ns, sizeof(long long));
  p->sub_stream = (int*)calloc((size_t)ns, sizeof(int));
  p->sub_work = (double*)calloc((size_t)ns, sizeof(double));
  if (!p->sub || !p->sub_off || !p->sub_stream || !p->sub_work)
    return fail(GFC_ERR_ALLOC, "gfc_plan_create_ragged: host allocation failed");
  for (int j = 0; j < ns; ++j) {
    const gfc_item& it = items[fast_items[j]];
    gfc_plan_opts o;
    memset(&o, 0, sizeof(o));
    o.H = it.H; o.W = it.W; o.C = it.C; o.batch = 1; o.dtype = GFC_F32; o.pad = 4; o.streams = 1;
    gfc_status st = gfc_plan_create_ex(&p->sub[j], &o);
    if (st != GFC_OK) return st;
    p->nsub = j + 1;
    p->sub_off[j] = it.offset;
    p->sub_work[j] = (double)it.C * it.H * it.W;
  }
  return ragged_set_streams(p, 4);
}

extern "C" {

gfc_status gfc_plan_create_ragged(gfc_plan** out, int n, const gfc_item* items, gfc_dtype dtype) {
  clear_error();
  if (!out || !items || n < 1) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create_ragged: bad arguments (n=%d)", n);
  *out = nullptr;
  if (dtype != GFC_F32 && dtype != GFC_F16 && dtype != GFC_BF16)
    return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create_ragged: unknown dtype %d", (int)dtype);
  std::vector<int> fast_items, generic_items;
  int maxM = 0, maxN = 0, maxH = 0, maxW = 0;
  long long nfields = 0, rag_total = 0;
  for (int i = 0; i < n; ++i) {
    const gfc_item& it = items[i];
    if (it.C < 1 || it.offset < 0)
      return fail(GFC_ERR_INVALID_ARG, "gfc_plan_create_ragged: item %d has C=%d offset=%lld", i, it.C, it.offset);
    int M, N;
    gfc_status st = gfc_padded_size(it.H, it.W, 4, GFC_SIZE_SMOOTH, &M, &N);
    if (st != GFC_OK) return st;
    maxM = std::max(maxM, M); maxN = std::max(maxN, N); maxH = std::max(maxH, it.H); maxW = std::max(maxW, it.W);
    nfields += it.C;
    rag_total = std::max(rag_total, it.offset + (long long)it.C * it.H * it.W);
    const bool fast = dtype == GFC_F32 && getenv("GFC_FORCE_GENERIC") == nullptr &&
                      (fast_supported(M, N) || fast_rows_supported(N));
    if (fast) fast_items.push_back(i);
    else generic_items.push_back(i);
  }
  if (nfields > (1 << 24)) return fail(GFC_ERR_UNSUPPORTED, "gfc_plan_create_ragged: too many fields");
  gfc_plan* p = nullptr;
  if (!generic_items.empty()) {
    const int ng = (int)generic_items.size();
    gfc_item* gen = (gfc_item*)malloc((size_t)ng * sizeof(gfc_item));
    if (!gen) return fail(GFC_ERR_ALLOC, "gfc_plan_create_ragged: host allocation failed");
    for (int i = 0; i < ng; ++i) gen[i] = items[generic_items[i]];
    gfc_status st = create_ragged_generic(&p, ng, gen, dtype);
    free(gen);
    if (st != GFC_OK) return st;
  } else {
    p = (gfc_plan*)calloc(1, sizeof(gfc_plan));
    if (!p) return fail(GFC_ERR_ALLOC, "gfc_plan_create_ragged: host allocation failed");
    p->ragged = true;
    p->pad = 4;
    p->dtype = dtype;
    p->C = 1;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->dev_err, 0, sizeof(int));
    if (e != cudaSuccess) {
      gfc_status st = cuda_fail(e, "gfc_plan_create_ragged");
      destroy_plan(p);
      return st;
    }
  }
  // the query reports the largest torus over all items
  p->M = maxM; p->N = maxN; p->Nh = maxN / 2 + 1; p->H = maxH; p->W = maxW;
  p->rag_total = rag_total;
  gfc_status st = attach_subplans(p, fast_items, items);
  if (st != GFC_OK) {
    destroy_plan(p);
    return st;
  }
  *out = p;
  return GFC_OK;
}


gfc_status gfc_plan_create(gfc_plan** plan, int H, int W, int C, int batch, gfc_dtype dtype) {
  gfc_plan_opts o;
  memset(&o, 0, sizeof(o));
  o.H = H; o.W = W; o.C = C; o.batch = batch; o.dtype = dtype;
  return gfc_plan_create_ex(plan, &o);
}

gfc_status gfc_plan_set_stream(gfc_plan* plan, void* stream) {
  clear_error();
  if (!plan) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_set_stream: null plan");
  plan->stream = (cudaStream_t)stream;
  return GFC_OK;
}

gfc_status gfc_plan_padded_size(const gfc_plan* plan, int* M, int* N, int* pad) {
  clear_error();
  if (!plan) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_padded_size: null plan");
  if (M) *M = plan->M;
  if (N) *N = plan->N;
  if (pad) *pad = plan->pad;
  return GFC_OK;
}

gfc_status gfc_plan_copy_green(const gfc_plan* plan, float* host_out) {
  clear_error();
  if (!plan || !host_out) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_copy_green: null argument");
  GFC_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  GFC_CUDA_TRY(cudaMemcpy(host_out, plan->G, (size_t)plan->M * plan->Nh * sizeof(float), cudaMemcpyDeviceToHost));
  return GFC_OK;
}

gfc_status gfc_plan_sync(gfc_plan* plan) {
  clear_error();
  if (!plan) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_sync: null plan");
  for (int j = 0; j < plan->nsub; ++j)
    if (gfc_status st = gfc_plan_sync(plan->sub[j])) return st;
  GFC_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  int h = 0;
  GFC_CUDA_TRY(cudaMemcpy(&h, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    cudaMemset(plan->dev_err, 0, sizeof(int));
    return fail(GFC_ERR_TIMEOUT, "gfc_plan_sync: device reported error code %d", h);
  }
  return GFC_OK;
}

}  // extern "C"

// (Re)assign a ragged plan's sub-plans to `k` internal streams: items in
// decreasing size, each to the stream with the least work so far.
gfc_status gfc::ragged_set_streams(gfc_plan* p, int k) {
  if (k < 1) k = 1;
  if (k > kMaxRagStreams) k = kMaxRagStreams;
  if (k > p->nsub) k = p->nsub;
  if (k < 1) k = 1;
  for (int s = p->rag_streams; s < k; ++s) {  // create the streams this needs beyond those there
    GFC_CUDA_TRY(cudaStreamCreateWithFlags(&p->rag_stream[s], cudaStreamNonBlocking));
    GFC_CUDA_TRY(cudaEventCreateWithFlags(&p->rag_done[s], cudaEventDisableTiming));
  }
  if (p->rag_streams < k) p->rag_streams = k;
  if (!p->rag_fork) GFC_CUDA_TRY(cudaEventCreateWithFlags(&p->rag_fork, cudaEventDisableTiming));
  int* order = (int*)malloc((size_t)p->nsub * sizeof(int));
  if (!order) return fail(GFC_ERR_ALLOC, "gfc_plan_create_ragged: host allocation failed");
  for (int j = 0; j < p->nsub; ++j) {  // insertion sort, largest item first (stable)
    int i = j;
    while (i > 0 && p->sub_work[order[i - 1]] < p->sub_work[j]) {
      order[i] = order[i - 1];
      --i;
    }
    order[i] = j;
  }
  double load[kMaxRagStreams] = {};
  for (int i = 0; i < p->nsub; ++i) {
    const int j = order[i];
    int best = 0;
    for (int s2 = 1; s2 < k; ++s2)
      if (load[s2] < load[best]) best = s2;
    p->sub_stream[j] = best;
    load[best] += p->sub_work[j];
  }
  free(order);
  p->rag_active = k;
  return GFC_OK;
}

static void destroy_plan(gfc_plan* p) {
  if (!p) return;
  for (int j = 0; j < p->nsub; ++j) destroy_plan(p->sub[j]);
  free(p->sub);
  free(p->sub_off);
  free(p->sub_stream);
  free(p->sub_work);
  for (int s = 0; s < p->rag_streams; ++s) {
    if (p->rag_stream[s]) cudaStreamDestroy(p->rag_stream[s]);
    if (p->rag_done[s]) cudaEventDestroy(p->rag_done[s]);
  }
  if (p->rag_fork) cudaEventDestroy(p->rag_fork);
  release_host_state(p);
  cudaFree(p->G);
  cudaFree(p->GT);
  cudaFree(p->d_desc);
  cudaFree(p->d_plans);
  free(p->chunk_begin);
  cudaFree(p->zbuf);
  cudaFree(p->twN);
  cudaFree(p->twM);
  cudaFree(p->spec);
  cudaFree(p->partial);
  cudaFree(p->edit_t2);
  cudaFree(p->colcoef);
  cudaFree(p->colcoef_h);
  cudaFree(p->powc_h);
  cudaFree(p->powc);
  cudaFree(p->tri_buf);
  exact_release(p);
  for (int sl = 0; sl < kMaxSlots; ++sl) {
    if (p->slot_stream[sl]) cudaStreamDestroy(p->slot_stream[sl]);
    if (p->slot_done[sl]) cudaEventDestroy(p->slot_done[sl]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  cudaFree(p->dev_err);
  free(p);
}

extern "C" {

gfc_status gfc_destroy(gfc_plan* p) {
  clear_error();
  destroy_plan(p);
  return GFC_OK;
}

}  // extern "C"

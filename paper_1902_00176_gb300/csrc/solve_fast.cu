// solve_fast.cu -- registry of the padded sizes with register-resident passes
// (kernels in fast_kernels.cuh, one translation unit per size pair).
#include "gfc_internal.h"

namespace gfc {

#define GFC_FAST_SHAPE(M, N)                                                                                  \
  cudaError_t fast_run_##M##x##N(gfc_plan*, const Bufs&, int, const void*, const void*, void*, void*, int, \
                                 cudaStream_t, const EditArgs*);                                          \
  size_t fast_zbuf_##M##x##N(int H);                                                                     \
  int fast_items_##M##x##N();
GFC_FAST_SHAPE(810, 1250)
GFC_FAST_SHAPE(1050, 1568)
GFC_FAST_SHAPE(270, 270)
GFC_FAST_SHAPE(72, 108)
#undef GFC_FAST_SHAPE

// row lengths compiled on their own (rows_family_*.cu)
#define GFC_ROW_LEN(N)                                                                                         \
  cudaError_t fast_rows_run_##N(gfc_plan*, const Bufs&, int, const void*, const void*, void*, void*, int,     \
                                cudaStream_t, const EditArgs*);                                               \
  size_t fast_rows_zbuf_##N(int H);                                                                            \
  int fast_rows_items_##N();
#define GFC_ROW_LENS(X)                                                                                          \
  X(140) X(160) X(180) X(200) X(224) X(252) X(294) X(320) X(360) X(400) X(448) X(500) X(560) X(630) X(700)     \
  X(784) X(882) X(980) X(1080) X(1120) X(1200) X(1372) X(1400) X(1536) X(1750) X(1960) X(2058)
GFC_ROW_LENS(GFC_ROW_LEN)
#undef GFC_ROW_LEN

namespace {
struct FastEntry {
  int M, N;
  cudaError_t (*run)(gfc_plan*, const Bufs&, int, const void*, const void*, void*, void*, int, cudaStream_t,
                     const EditArgs*);
  size_t (*zbuf)(int H);
  int (*items)();
};
const FastEntry kFast[] = {
    {810, 1250, fast_run_810x1250, fast_zbuf_810x1250, fast_items_810x1250},
    {1050, 1568, fast_run_1050x1568, fast_zbuf_1050x1568, fast_items_1050x1568},
    {270, 270, fast_run_270x270, fast_zbuf_270x270, fast_items_270x270},
    {72, 108, fast_run_72x108, fast_zbuf_72x108, fast_items_72x108},
};
const FastEntry* find(int M, int N) {
  for (const FastEntry& e : kFast)
    if (e.M == M && e.N == N) return &e;
  return nullptr;
}
struct RowEntry {
  int N;
  cudaError_t (*run)(gfc_plan*, const Bufs&, int, const void*, const void*, void*, void*, int, cudaStream_t,
                     const EditArgs*);
  size_t (*zbuf)(int H);
  int (*items)();
};
#define GFC_ROW_ENTRY(N) {N, fast_rows_run_##N, fast_rows_zbuf_##N, fast_rows_items_##N},
const RowEntry kRows[] = {GFC_ROW_LENS(GFC_ROW_ENTRY)};
#undef GFC_ROW_ENTRY
const RowEntry* find_rows(int N) {
  for (const RowEntry& e : kRows)
    if (e.N == N) return &e;
  return nullptr;
}
}  // namespace

bool fast_supported(int M, int N) { return find(M, N) != nullptr; }

bool fast_rows_supported(int N) { return find_rows(N) != nullptr; }

int fast_row_lengths(int* out, int cap) {  // the listed lengths that have a kernel set
  int m = 0;
  for (int r : kRowLengthList) {
    bool found = find_rows(r) != nullptr;
    for (const FastEntry& e : kFast) found = found || e.N == r;
    if (!found) continue;
    if (m < cap) out[m] = r;
    ++m;
  }
  return m;
}

size_t fast_zbuf_elems(int H, int M, int N) {
  if (const FastEntry* e = find(M, N)) return e->zbuf(H);
  if (const RowEntry* r = find_rows(N)) return r->zbuf(H);
  return 0;
}

int fast_row_items(int M, int N) {
  if (const FastEntry* e = find(M, N)) return e->items();
  if (const RowEntry* r = find_rows(N)) return r->items();
  return 0;
}

cudaError_t run_chunk_fast(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                           void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  if (const FastEntry* e = find(P->M, P->N)) return e->run(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
  if (const RowEntry* r = find_rows(P->N)) return r->run(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
  return cudaErrorNotSupported;
}

}  // namespace gfc

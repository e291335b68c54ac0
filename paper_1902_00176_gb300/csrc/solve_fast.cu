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
}  // namespace

bool fast_supported(int M, int N) { return find(M, N) != nullptr; }

size_t fast_zbuf_elems(int H, int M, int N) {
  const FastEntry* e = find(M, N);
  return e ? e->zbuf(H) : 0;
}

int fast_row_items(int M, int N) {
  const FastEntry* e = find(M, N);
  return e ? e->items() : 0;
}

cudaError_t run_chunk_fast(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                           void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  const FastEntry* e = find(P->M, P->N);
  if (!e) return cudaErrorNotSupported;
  return e->run(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
}

}  // namespace gfc

// rows_family.cuh -- register-resident row passes for one row length N, for
// plans whose column direction runs the recursive column solve (no column
// kernels are compiled for these lengths; see run_rows_shape). Each
// rows_family_<k>.cu instantiates a few lengths so the library builds in
// parallel; solve_fast.cu lists them.
#pragma once

#include "fast_kernels.cuh"

// One row length: N = R1 R2 with R2 threads per transform and F transforms per
// block (about 128 threads, within the shared memory of 2 forward blocks and 3
// inverse blocks per SM, 4 and 4 for N <= 512).
#define GFC_ROW_SHAPE(N_, R1_, R2_, F_)                                                                          \
  using RowF_##N_ = RowShape<N_, R1_, R2_, F_>;                                                                 \
  cudaError_t fast_rows_run_##N_(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1,       \
                                 void* out0, void* out1, int nf, cudaStream_t st, const EditArgs* ed) {         \
    return run_rows_shape<RowF_##N_>(P, bf, mode, in0, in1, out0, out1, nf, st, ed);                             \
  }                                                                                                             \
  size_t fast_rows_zbuf_##N_(int H) { return fast_zbuf_elems_for<RowF_##N_>(H); }                               \
  int fast_rows_items_##N_() { return F_; }

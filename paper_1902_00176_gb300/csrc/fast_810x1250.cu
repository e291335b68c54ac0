// fast_810x1250.cu -- register-resident passes for the 810 x 1250 padded domain
// (row schedule RowShape<1250, 50, 25, 5>, column schedule ColShape<810, 27, 30, 8>).
#include "fast_kernels.cuh"

namespace gfc {

using RowS_810x1250 = RowShape<1250, 50, 25, 5>;
using ColS_810x1250 = ColShape<810, 27, 30, 8>;

cudaError_t fast_run_810x1250(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                          void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  return run_fast_shape<RowS_810x1250, ColS_810x1250>(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
}

size_t fast_zbuf_810x1250(int H) { return fast_zbuf_elems_for<RowS_810x1250>(H); }

int fast_items_810x1250() { return RowS_810x1250::F; }

}  // namespace gfc
